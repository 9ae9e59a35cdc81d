// sidm_api.cu -- C ABI of libsidm: context, cell build (a0), scatter resolve
// (a4), energy/momentum reduction (a5), harness kernels, and the host-side
// FP64 quadrature that fills the Lambda lookup table.
//
// Paper: Fischer, Yu & Dolag (2025).  Sect. 2 (spline kernel, N_ngb-adaptive
// kernel size, explicit energy and momentum conservation), Sect. 3.5 (the
// geometric factor Lambda of the interaction probability), Sect. 5
// (conservation independent of the kernel).
#include <algorithm>
#include <mutex>
#include <vector>
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "sidm_internal.cuh"
#include "sidm_sum.cuh"
#include "sidm_sort.cuh"

using namespace sidm;

namespace {

thread_local std::string g_create_err;

constexpr int kChunk = 16384;        // particles per reduction chunk

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ int halo_of(const int64_t* __restrict__ off, int H, int64_t s)
{
    int lo = 0, hi = H - 1;               // largest h with off[h] <= s
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= s) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int bsearch32(const int32_t* __restrict__ off, int H, int32_t s)
{
    int lo = 0, hi = H - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= s) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ unsigned long long spread3(uint32_t v)
{
    unsigned long long x = v & 0x1FFFFFu;
    x = (x | (x << 32)) & 0x1F00000000FFFFull;
    x = (x | (x << 16)) & 0x1F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ uint32_t compact3(unsigned long long x)
{
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10C30C30C30C30C3ull;
    x = (x ^ (x >> 4)) & 0x100F00F00F00F00Full;
    x = (x ^ (x >> 8)) & 0x1F0000FF0000FFull;
    x = (x ^ (x >> 16)) & 0x1F00000000FFFFull;
    x = (x ^ (x >> 32)) & 0x1FFFFFull;
    return (uint32_t)x;
}

// ------------------------------------------------------------------ a0 kernels
// Per-halo bounding box: exact min/max of the FP64 positions as integer
// min/max of their order-preserving bit images (integer pipes, not FP64).
// kBboxSplit CTAs per reduction chunk, each a quarter of it with all its loads
// in flight; one atomic per CTA and bound.
constexpr int kBboxSplit = 4;
__global__ void __launch_bounds__(256) k_bbox(const double* __restrict__ pos, int64_t N,
                                              const int32_t* __restrict__ chunk_halo,
                                              const int64_t* __restrict__ chunk_begin,
                                              const int64_t* __restrict__ halo_off, int H,
                                              unsigned long long* __restrict__ bb)
{
    __shared__ unsigned long long red[8][6];
    const int c = blockIdx.x / kBboxSplit, part = blockIdx.x % kBboxSplit;
    const int h = chunk_halo[c];
    int64_t b = chunk_begin[c];
    int64_t e = b + kChunk;
    if (e > halo_off[h + 1]) e = halo_off[h + 1];
    b += (int64_t)part * (kChunk / kBboxSplit);
    if (b + kChunk / kBboxSplit < e) e = b + kChunk / kBboxSplit;
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
#pragma unroll 4
    for (int64_t s = b + threadIdx.x; s < e; s += blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const unsigned long long v = dbl_to_ord(pos[a * N + s]);
            mn[a] = min(mn[a], v);
            mx[a] = max(mx[a], v);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = min(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int a = 0; a < 3; ++a) { red[warp][a] = mn[a]; red[warp][3 + a] = mx[a]; }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int a = threadIdx.x;
        unsigned long long v = red[0][a];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = a < 3 ? min(v, red[w][a]) : max(v, red[w][a]);
        if (b < e) {                                      // a part past the halo's end has nothing
            if (a < 3) atomicMin(&bb[a * H + h], v);
            else atomicMax(&bb[a * H + h], v);
        }
    }
}

// Halo frame: 2^E > largest extent, O = floor(min / 2^E) 2^E per axis.
__global__ void k_frame(int H, const int64_t* __restrict__ halo_off, const unsigned long long* __restrict__ bb,
                        HaloFrame* __restrict__ fr)
{
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= H) return;
    HaloFrame f;
    double mn[3], ext = 0.0;
    const bool empty = halo_off[h + 1] == halo_off[h];
    for (int a = 0; a < 3; ++a) {
        mn[a] = empty ? 0.0 : ord_to_dbl(bb[a * H + h]);
        double mx = empty ? 0.0 : ord_to_dbl(bb[(3 + a) * H + h]);
        ext = fmax(ext, mx - mn[a]);
    }
    int E = 0;
    if (ext > 0.0) frexp(ext, &E);           // ext = m 2^E, m in [1/2, 1)
    for (int a = 0; a < 3; ++a) f.O[a] = ldexp(floor(ldexp(mn[a], -E)), E);
    f.E = E;
    f.qs = ldexp(1.0, kMortonBits - E - 1);
    f.cube = (float)ldexp(1.0, E + 1);
    f.margin = (float)ldexp(1.0, E + 1 - 20);
    f.fine = (float)ldexp(1.0, E + 1 - kMortonBits);
    fr[h] = f;
}

// floor(t 2^(17-E-1)) clamped to [0, 2^17 - 1], t = RN(x - O) in FP64: the
// scaling by a power of two is exact, so the floor is read off t's bits
// (t = M 2^(e-52), M the integer significand): M >> (36 + E - e), 0 for a
// shift of 64 or more, the clamp for a negative one.  Only the subtraction
// runs on the FP64 pipe.
__device__ __forceinline__ uint32_t morton_coord(double x, double O, int E)
{
    const uint32_t qmax = (1u << kMortonBits) - 1u;
    const double t = __dsub_rn(x, O);
    const unsigned long long b = (unsigned long long)__double_as_longlong(t);
    const int eb = (int)((b >> 52) & 2047ull);
    const unsigned long long mant = b & ((1ull << 52) - 1ull);
    if (b >> 63) return 0u;                                  // t <= 0 (or a negative NaN)
    if (eb == 2047) return mant ? 0u : qmax;                 // NaN: 0, +inf: the clamp
    const unsigned long long M = eb ? (mant | (1ull << 52)) : mant;
    const int sh = 36 + E - ((eb ? eb : 1) - 1023);
    if (sh >= 64) return 0u;
    if (sh < 0) return qmax;
    const unsigned long long fl = M >> sh;
    return fl >= qmax ? qmax : (uint32_t)fl;
}

// Sort key = halo << 51 | Morton(q), q = floor((x - O) 2^(17-E-1)) clamped;
// the digit counts of every sort pass taken on the way (hist [passes][256],
// zero on entry).
__global__ void __launch_bounds__(256) k_keys(const double* __restrict__ pos, int64_t N,
                                              const int64_t* __restrict__ halo_off, int H,
                                              const HaloFrame* __restrict__ fr, unsigned long long* __restrict__ key,
                                              uint32_t* __restrict__ val, int passes, uint32_t* __restrict__ hist)
{
    __shared__ uint32_t sh[sidm_sort::kMaxPasses][256];
    for (int i = threadIdx.x; i < sidm_sort::kMaxPasses * 256; i += blockDim.x) (&sh[0][0])[i] = 0u;
    __syncthreads();
    // two particles per thread and trip, their six loads issued together
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s0 < N; s0 += 2 * stride) {
        double x[2][3];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t s = s0 + u * stride;
#pragma unroll
            for (int a = 0; a < 3; ++a) x[u][a] = s < N ? pos[a * N + s] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t s = s0 + u * stride;
            if (s >= N) break;
            const int h = H == 1 ? 0 : halo_of(halo_off, H, s);
            const HaloFrame& f = fr[h];
            const uint32_t q0 = morton_coord(x[u][0], f.O[0], f.E);
            const uint32_t q1 = morton_coord(x[u][1], f.O[1], f.E);
            const uint32_t q2 = morton_coord(x[u][2], f.O[2], f.E);
            const unsigned long long k =
                ((unsigned long long)h << kHaloShift) | spread3(q0) | (spread3(q1) << 1) | (spread3(q2) << 2);
            key[s] = k;
            val[s] = (uint32_t)s;
            sidm_sort::count_digits(sh, k, passes);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) {
        const uint32_t v = (&sh[0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
}

// Leaf bookkeeping: halo of each leaf, and its frame origin = corner of the
// finest Morton cell of its first particle (relative to O, exact in FP32);
// cellb = RN64(O + origin) per axis, the base the gather subtracts.
__global__ void k_leaf_fill(int L, int H, const int32_t* __restrict__ leaf_off, const int64_t* __restrict__ halo_off,
                            const unsigned long long* __restrict__ skey, const HaloFrame* __restrict__ fr,
                            int32_t* __restrict__ leaf_halo, float4* __restrict__ cell, double4* __restrict__ cellb)
{
    int leaf = blockIdx.x * blockDim.x + threadIdx.x;
    if (leaf >= L) return;
    const int h = bsearch32(leaf_off, H, leaf);
    leaf_halo[leaf] = h;
    const int64_t s = halo_off[h] + (int64_t)(leaf - leaf_off[h]) * kLeaf;
    const unsigned long long k = skey[s] & ((1ull << kHaloShift) - 1ull);
    const float fine = fr[h].fine;
    const float4 c = make_float4((float)compact3(k) * fine, (float)compact3(k >> 1) * fine,
                                 (float)compact3(k >> 2) * fine, 0.f);
    cell[leaf] = c;
    const HaloFrame& f = fr[h];
    cellb[leaf] = make_double4(__dadd_rn(f.O[0], (double)c.x), __dadd_rn(f.O[1], (double)c.y),
                               __dadd_rn(f.O[2], (double)c.z), 0.0);
}

// Gather into Morton order (the FP64 form): sorted user arrays (scratch),
// internal padded tracks, permutation.
template <class R>
__global__ void k_gather(int64_t N, int H, const int64_t* __restrict__ halo_off, const int64_t* __restrict__ halo_pad,
                         const unsigned long long* __restrict__ skey,
                         const uint32_t* __restrict__ sval, const double* __restrict__ pos, const R* __restrict__ vel,
                         const uint32_t* __restrict__ id, double* __restrict__ tpos, R* __restrict__ tvel,
                         uint32_t* __restrict__ tid, uint32_t* __restrict__ perm,
                         typename Vec4<R>::T* __restrict__ P4, uint32_t* __restrict__ ID, DevCounters* cnt,
                         const R* __restrict__ hprev)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t src = sval[s];
        const int h = (int)(skey[s] >> kHaloShift);
        const int64_t local = s - halo_off[h];
        const int64_t slot = halo_pad[h] + local;
        double x[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            x[a] = pos[a * N + src];
            tpos[a * N + s] = x[a];
            tvel[a * N + s] = vel[a * N + src];
        }
        const uint32_t myid = id[src];
        tid[s] = myid;
        perm[s] = src;
        ID[slot] = myid;
        if (myid >= kIdLimit || !isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2]))
            raise_status(cnt, SIDM_DEV_BAD_INPUT);
        typename Vec4<R>::T p;
        p.x = (R)x[0]; p.y = (R)x[1]; p.z = (R)x[2];
        p.w = hprev ? hprev[src] : R(0);   // previous kernel size: a guess for the search
        P4[slot] = p;
    }
}

// The mixed form's gather, one warp per leaf (slot = leaf * 32 + lane), with
// the leaf's bounding box in the halo frame taken on the way: each point
// cell + offset is added with rounding down and up (no FP64), so the box holds
// it exactly (the canonical positions the kernels test against it lie within a
// few FP32 ulps, far inside the pruning margin).  Same writes as k_gather<R,
// true> followed by k_leaf_bbox_p4, without reading the padded track back.
template <class R>
__global__ void __launch_bounds__(256) k_gather_leaves(int L, int64_t N, const int32_t* __restrict__ leaf_halo,
                                                       const int32_t* __restrict__ leaf_off,
                                                       const int64_t* __restrict__ halo_off,
                                                       const float4* __restrict__ cell,
                                                       const double4* __restrict__ cellb,
                                                       const uint32_t* __restrict__ sval, const double* __restrict__ pos,
                                                       const R* __restrict__ vel, const uint32_t* __restrict__ id,
                                                       double* __restrict__ tpos, R* __restrict__ tvel,
                                                       uint32_t* __restrict__ tid, uint32_t* __restrict__ perm,
                                                       typename Vec4<R>::T* __restrict__ P4, uint32_t* __restrict__ ID,
                                                       DevCounters* cnt, const R* __restrict__ hprev,
                                                       float4* __restrict__ nlo, float4* __restrict__ nhi)
{
    const int lane = threadIdx.x & 31;
    const int leaf = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (leaf >= L) return;                                     // whole warps
    const int h = leaf_halo[leaf];
    const int64_t local = (int64_t)(leaf - leaf_off[h]) * kLeaf + lane;
    const float4 c = cell[leaf];
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (local < halo_off[h + 1] - halo_off[h]) {
        const int64_t s = halo_off[h] + local;
        const int64_t slot = (int64_t)leaf * kLeaf + lane;
        const uint32_t src = sval[s];
        double x[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            x[a] = pos[a * N + src];
            tpos[a * N + s] = x[a];
            tvel[a * N + s] = vel[a * N + src];
        }
        const uint32_t myid = id[src];
        tid[s] = myid;
        perm[s] = src;
        ID[slot] = myid;
        if (myid >= kIdLimit || !isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2]))
            raise_status(cnt, SIDM_DEV_BAD_INPUT);
        const double4 b = cellb[leaf];
        typename Vec4<R>::T p;
        p.x = (R)__double2float_rn(__dsub_rn(x[0], b.x));
        p.y = (R)__double2float_rn(__dsub_rn(x[1], b.y));
        p.z = (R)__double2float_rn(__dsub_rn(x[2], b.z));
        p.w = hprev ? hprev[src] : R(0);   // previous kernel size: a guess for the search
        P4[slot] = p;
        mn[0] = __fadd_rd(c.x, (float)p.x); mn[1] = __fadd_rd(c.y, (float)p.y); mn[2] = __fadd_rd(c.z, (float)p.z);
        mx[0] = __fadd_ru(c.x, (float)p.x); mx[1] = __fadd_ru(c.y, (float)p.y); mx[2] = __fadd_ru(c.z, (float)p.z);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    if (lane == 0) {
        nlo[leaf] = make_float4(mn[0], mn[1], mn[2], 0.f);
        nhi[leaf] = make_float4(mx[0], mx[1], mx[2], 0.f);
    }
}

// Leaf bounding boxes in the halo frame (FP32, rounded outward) from the FP64
// positions (the FP64 form); one warp per leaf.
__global__ void k_leaf_bbox(int L, int64_t N, const int32_t* __restrict__ leaf_halo, const int32_t* __restrict__ leaf_off,
                            const int64_t* __restrict__ halo_off, const HaloFrame* __restrict__ fr,
                            const double* __restrict__ pos, float4* __restrict__ nlo, float4* __restrict__ nhi)
{
    const int lane = threadIdx.x & 31;
    const int leaf = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (leaf >= L) return;
    const int h = leaf_halo[leaf];
    const int64_t b = halo_off[h] + (int64_t)(leaf - leaf_off[h]) * kLeaf;
    int64_t e = b + kLeaf; if (e > halo_off[h + 1]) e = halo_off[h + 1];
    const HaloFrame f = fr[h];
    const int64_t s = b + lane < e ? b + lane : b;
    // rounding down (up) is monotone, so the FP32 minimum of the rounded-down
    // offsets is the rounded-down FP64 minimum: the reduction runs in FP32
    float mn[3], mx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double y = __dsub_rn(pos[a * N + s], f.O[a]);
        mn[a] = __double2float_rd(y);
        mx[a] = __double2float_ru(y);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    if (lane == 0) {
        nlo[leaf] = make_float4(mn[0], mn[1], mn[2], 0.f);
        nhi[leaf] = make_float4(mx[0], mx[1], mx[2], 0.f);
    }
}

// Max kernel size per leaf (into lo.w), from the padded h track.
// SIDM time step and power-of-two bin of every particle from its summed pair
// probabilities; the halo minimum by an atomic min on order-preserving bits.
__global__ void k_timestep(int64_t N, int H, const int64_t* __restrict__ halo_off, const float* __restrict__ sump,
                           const double* __restrict__ dt, double tau, double dt_min, double dt_max, int n_bins,
                           double* __restrict__ dt_out, int32_t* __restrict__ bin_out,
                           unsigned long long* __restrict__ halo_min)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < N; u += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = H - 1;                    // halo of particle u: last h with halo_off[h] <= u
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (halo_off[mid] <= u) lo = mid; else hi = mid - 1;
        }
        const double sp = (double)sump[u];
        double di = sp > 0.0 ? tau * dt[lo] / sp : dt_max;
        di = fmin(fmax(di, dt_min), dt_max);
        int b = 0;
        while (b < n_bins - 1 && ldexp(dt_max, -b) > di) ++b;
        if (dt_out) dt_out[u] = di;
        if (bin_out) bin_out[u] = b;
        if (halo_min) atomicMin(halo_min + lo, dbl_to_ord(di));
    }
}

__global__ void k_halo_min_final(int H, const unsigned long long* __restrict__ ord, double dt_max, double* __restrict__ out)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h < H) out[h] = ord[h] == ~0ull ? dt_max : ord_to_dbl(ord[h]);
}

// sigma_eff / s0 = (1/6) int_0^inf t^3 e^-t / (1 + beta t)^2 dt, beta = 4 nu^2 / w^2
// (the Maxwellian average <v^5 sigma(v)> / <v^5> with t = v^2 / (4 nu^2)):
// 4-point Gauss-Legendre on 48 panels with edges 64 (k/48)^2, which follow the
// 1/beta scale near t = 0; error below 1e-6 up to beta = 1e4.  Evaluated in
// the form's precision (FP32 in the mixed form, whose outputs are FP32).
template <class R>
__device__ R sigma_eff_ratio(R beta)
{
    const R a = sqrt(R(3) / R(7) + R(2) / R(7) * sqrt(R(1.2))), b = sqrt(R(3) / R(7) - R(2) / R(7) * sqrt(R(1.2)));
    const R wa = (R(18) - sqrt(R(30))) / R(36), wb = (R(18) + sqrt(R(30))) / R(36);
    const R xg[4] = {-a, -b, b, a}, wg[4] = {wa, wb, wb, wa};
    R tot = R(0);
    for (int k = 0; k < 48; ++k) {
        const R lo = R(64) * (R(k) / R(48)) * (R(k) / R(48)), hi = R(64) * (R(k + 1) / R(48)) * (R(k + 1) / R(48));
        const R c = R(0.5) * (lo + hi), hw = R(0.5) * (hi - lo);
        for (int g = 0; g < 4; ++g) {
            const R t = c + hw * xg[g];
            const R den = R(1) + beta * t;
            tot += hw * wg[g] * t * t * t * exp(-t) / (den * den);
        }
    }
    return tot / R(6);
}

// Local diagnostics from the kernel-weighted pair moments plus the self term
// (one thread per slot of a leaf).
template <class R>
__global__ void k_diag_final(int L, const int32_t* __restrict__ leaf_halo, const int32_t* __restrict__ leaf_off,
                             const int64_t* __restrict__ halo_off, const typename Vec4<R>::T* __restrict__ P4,
                             const typename Vec4<R>::T* __restrict__ V4, const double* __restrict__ dacc, int64_t N,
                             const double* __restrict__ mass, const sidm_xs* __restrict__ xs,
                             const int32_t* __restrict__ ngb, double G, R* __restrict__ out)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int leaf = (int)(t / kLeaf), lane = (int)(t % kLeaf);
    if (leaf >= L) return;
    const int h = leaf_halo[leaf];
    const int64_t local = (int64_t)(leaf - leaf_off[h]) * kLeaf + lane;
    if (local >= halo_off[h + 1] - halo_off[h]) return;
    const int64_t u = halo_off[h] + local;
    const int64_t slot = (int64_t)leaf * kLeaf + lane;
    const double hv = (double)P4[slot].w;
    const typename Vec4<R>::T v = V4[slot];
    const double vx = (double)v.x, vy = (double)v.y, vz = (double)v.z;
    const double m = mass[h];
    const double w0 = m * (8.0 / 3.14159265358979323846) / (hv * hv * hv);
    const double sw = dacc[u] + w0;
    const double mx = (dacc[N + u] + w0 * vx) / sw, my = (dacc[2 * N + u] + w0 * vy) / sw,
                 mz = (dacc[3 * N + u] + w0 * vz) / sw;
    const double m2 = (dacc[4 * N + u] + w0 * (vx * vx + vy * vy + vz * vz)) / sw;
    const double nu = sqrt(fmax((m2 - (mx * mx + my * my + mz * mz)) / 3.0, 0.0));
    const sidm_xs x = xs[h];
    const double se = x.kind == 1 ? x.s0 * (double)sigma_eff_ratio<R>((R)(4.0 * nu * nu / (x.w * x.w))) : x.s0;
    const double rho = sw;
    out[u] = (R)rho;
    out[N + u] = (R)nu;
    out[2 * N + u] = (R)se;
    out[3 * N + u] = (R)(se * cbrt(rho * rho) * cbrt(3.0 * m * ngb[h] / (3.14159265358979323846 * sqrt(2.0))));
    out[4 * N + u] = (R)(sqrt(4.0 * 3.14159265358979323846 * G / (rho * nu * nu)) / se);
}

template <class R>
__global__ void k_leaf_hmax(int L, int H, const int32_t* __restrict__ leaf_halo, const int32_t* __restrict__ leaf_off,
                            const int64_t* __restrict__ halo_off, const typename Vec4<R>::T* __restrict__ P4,
                            float4* __restrict__ nlo)
{
    const int lane = threadIdx.x & 31;
    const int leaf = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (leaf >= L) return;
    const int h = leaf_halo[leaf];
    const int64_t local0 = (int64_t)(leaf - leaf_off[h]) * kLeaf;
    const int cntl = (int)min((int64_t)kLeaf, halo_off[h + 1] - halo_off[h] - local0);
    float m = 0.f;
    if (lane < cntl) {
        const R hv = P4[(int64_t)leaf * kLeaf + lane].w;
        m = (float)hv;
        if ((R)m < hv) m = __uint_as_float(__float_as_uint(m) + 1u);   // round up
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) nlo[leaf].w = m;
}

// One tree level: union of up to kArity children (bbox and max h).
__global__ void __launch_bounds__(256) k_tree_level(int lev, int H, const int32_t* __restrict__ lvl_off,
                                                    float4* __restrict__ nlo, float4* __restrict__ nhi)
{
    // one warp per node, one child per lane (kArity == 32): every child's box
    // is loaded at once, then min/max across the warp
    static_assert(kArity == 32, "one child per lane");
    const int32_t* off = lvl_off + lev * (H + 1);
    const int32_t* coff = lvl_off + (lev - 1) * (H + 1);
    const int total = off[H] - off[0];
    const int lane = threadIdx.x & 31;
    const int t = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (t >= total) return;                                  // whole warps
    const int node = off[0] + t;
    const int h = bsearch32(off, H, node);
    const int local = node - off[h];
    const int c = coff[h] + local * kArity + lane;
    float4 lo = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
    float4 hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
    if (c < coff[h + 1]) { lo = nlo[c]; hi = nhi[c]; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
        lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
        lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o));
        lo.w = fmaxf(lo.w, __shfl_xor_sync(0xffffffffu, lo.w, o));
        hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
        hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
        hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o));
    }
    if (lane == 0) {
        nlo[node] = lo;
        nhi[node] = make_float4(hi.x, hi.y, hi.z, 0.f);
    }
}

// ------------------------------------------------------------------ a2 prep
template <class R>
__global__ void k_vel_refresh(int64_t N, int H, const int64_t* __restrict__ halo_off, const int64_t* __restrict__ halo_pad,
                              const R* __restrict__ vel, const uint32_t* __restrict__ ID,
                              typename Vec4<R>::T* __restrict__ V4)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
        const int h = halo_of(halo_off, H, s);
        const int64_t slot = halo_pad[h] + (s - halo_off[h]);
        typename Vec4<R>::T v;
        v.x = vel[s]; v.y = vel[N + s]; v.z = vel[2 * N + s];
        if (sizeof(R) == 4) v.w = (R)__uint_as_float(ID[slot]);
        else v.w = (R)ID[slot];
        V4[slot] = v;
    }
}

// ------------------------------------------------------------------ a4 resolve
// 128-bit fixed-point accumulation (units of 2^-80) of a double; integer
// additions commute, so the sum does not depend on the order of the events.
__device__ __forceinline__ void fx_add(DevCounters* cnt, double v)
{
    const double hi_d = floor(ldexp(v, 16));                 // v 2^80 / 2^64
    const double lo_d = ldexp(v, 80) - ldexp(hi_d, 64);      // in [0, 2^64)
    unsigned long long lo = lo_d >= 18446744073709551615.0 ? 0xFFFFFFFFFFFFFFFFull : __double2ull_rz(lo_d);
    unsigned long long hi = (unsigned long long)(long long)hi_d;
    unsigned long long old = atomicAdd(&cnt->de_lo, lo);
    if (old + lo < old) hi += 1ull;
    atomicAdd(&cnt->de_hi, hi);
}

// Isotropic scatter of event E (Sect. 2, reading C6) on the current velocities
// (read and written through L2); returns the change of the pair's kinetic
// energy from the stored values, in FP64.  Equal masses within a halo.
template <class R>
__device__ __forceinline__ double apply_isotropic(const sidm_event& E, R* vel, int64_t N, const double* __restrict__ mass)
{
    R* vx = vel; R* vy = vel + N; R* vz = vel + 2 * N;
    const int h = (int)(E.key >> 54);
    const double m = mass[h];
    const R vi[3] = {__ldcg(vx + E.i), __ldcg(vy + E.i), __ldcg(vz + E.i)};
    const R vj[3] = {__ldcg(vx + E.j), __ldcg(vy + E.j), __ldcg(vz + E.j)};
    R ct, st_, sp, cp;
    if (sizeof(R) == 4) {
        ct = (R)fmaf((float)E.x1, 0x1p-31f, -1.0f);
        st_ = (R)sqrtf(fmaxf(0.f, 1.f - (float)ct * (float)ct));
        float s_, c_;
        sincospif((float)E.x2 * 0x1p-31f, &s_, &c_);
        sp = (R)s_; cp = (R)c_;
    } else {
        ct = (R)(2.0 * ldexp((double)E.x1, -32) - 1.0);
        st_ = (R)sqrt(fmax(0.0, 1.0 - (double)ct * (double)ct));
        double s_, c_;
        sincospi(ldexp((double)E.x2, -31), &s_, &c_);
        sp = (R)s_; cp = (R)c_;
    }
    const R nh[3] = {st_ * cp, st_ * sp, ct};
    // equal masses within a halo: v_cm = (v_i + v_j)/2, weights 1/2
    R dv2 = R(0), vc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        vc[a] = R(0.5) * (vi[a] + vj[a]);
        const R d = vi[a] - vj[a];
        dv2 += d * d;
    }
    const R hw = R(0.5) * sqrt(dv2);
    R ni[3], nj[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) { ni[a] = vc[a] + hw * nh[a]; nj[a] = vc[a] - hw * nh[a]; }
    __stcg(vx + E.i, ni[0]); __stcg(vy + E.i, ni[1]); __stcg(vz + E.i, ni[2]);
    __stcg(vx + E.j, nj[0]); __stcg(vy + E.j, nj[1]); __stcg(vz + E.j, nj[2]);
    double e0 = 0.0, e1 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        e0 = __dadd_rn(e0, __dadd_rn(__dmul_rn((double)vi[a], (double)vi[a]), __dmul_rn((double)vj[a], (double)vj[a])));
        e1 = __dadd_rn(e1, __dadd_rn(__dmul_rn((double)ni[a], (double)ni[a]), __dmul_rn((double)nj[a], (double)nj[a])));
    }
    return __dmul_rn(0.5 * m, __dsub_rn(e1, e0));
}

// Forward-dominated interaction of record E (Sect. 3.8 with App. A, reading
// C20): the relative velocity u = v_i - v_j turns by alpha, cos(alpha) = 1 - D,
// sin(alpha) = sqrt(D (2 - D)), D = (sigma_V/m)/3 |u| G, G = m_j Lambda dt of the
// step start, towards the projection onto u's normal plane of the isotropic
// Philox direction of words 1 and 2 (uniform in azimuth about u); |u| and v_cm
// are kept.  D = 0 changes nothing.  Returns the pair's kinetic-energy change
// from the stored values (FP64).
template <class R>
__device__ __forceinline__ double apply_drag(const sidm_event& E, double G, const sidm_xs& xs, R* vel, int64_t N,
                                             const double* __restrict__ mass)
{
    R* vx = vel; R* vy = vel + N; R* vz = vel + 2 * N;
    const double m = mass[(int)(E.key >> 54)];
    const R vi[3] = {__ldcg(vx + E.i), __ldcg(vy + E.i), __ldcg(vz + E.i)};
    const R vj[3] = {__ldcg(vx + E.j), __ldcg(vy + E.j), __ldcg(vz + E.j)};
    R u[3], vc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) { u[a] = vi[a] - vj[a]; vc[a] = R(0.5) * (vi[a] + vj[a]); }
    const R un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    R sig = (R)xs.s0;
    if (xs.kind == 1) { const R q = un / (R)xs.w; const R t = R(1) + q * q; sig = (R)xs.s0 / (t * t); }
    const R D = sig / R(3) * un * (R)G;
    if (!(D > R(0))) return 0.0;
    R ca, sa;
    if (D < R(2)) { ca = R(1) - D; sa = sqrt(D * (R(2) - D)); } else { ca = R(-1); sa = R(0); }
    // the turn's direction: the isotropic Philox direction w (words 1, 2, as an
    // isotropic scatter draws it) projected onto the plane normal to u
    R ct, st_, sp, cp;
    if (sizeof(R) == 4) {
        ct = (R)fmaf((float)E.x1, 0x1p-31f, -1.0f);
        st_ = (R)sqrtf(fmaxf(0.f, 1.f - (float)ct * (float)ct));
        float s_, c_;
        sincospif((float)E.x2 * 0x1p-31f, &s_, &c_);
        sp = (R)s_; cp = (R)c_;
    } else {
        ct = (R)(2.0 * ldexp((double)E.x1, -32) - 1.0);
        st_ = (R)sqrt(fmax(0.0, 1.0 - (double)ct * (double)ct));
        double s_, c_;
        sincospi(ldexp((double)E.x2, -31), &s_, &c_);
        sp = (R)s_; cp = (R)c_;
    }
    const R w[3] = {st_ * cp, st_ * sp, ct};
    const R nh[3] = {u[0] / un, u[1] / un, u[2] / un};
    const R wn = w[0] * nh[0] + w[1] * nh[1] + w[2] * nh[2];
    R ep[3], el = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) { ep[a] = w[a] - wn * nh[a]; el += ep[a] * ep[a]; }
    el = sqrt(el);
    const R sc = el > R(0) ? un * sa / el : R(0);
    R ni[3], nj[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const R up = ca * u[a] + sc * ep[a];
        ni[a] = vc[a] + R(0.5) * up;
        nj[a] = vc[a] - R(0.5) * up;
    }
    __stcg(vx + E.i, ni[0]); __stcg(vy + E.i, ni[1]); __stcg(vz + E.i, ni[2]);
    __stcg(vx + E.j, nj[0]); __stcg(vy + E.j, nj[1]); __stcg(vz + E.j, nj[2]);
    double e0 = 0.0, e1 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        e0 = __dadd_rn(e0, __dadd_rn(__dmul_rn((double)vi[a], (double)vi[a]), __dmul_rn((double)vj[a], (double)vj[a])));
        e1 = __dadd_rn(e1, __dadd_rn(__dmul_rn((double)ni[a], (double)ni[a]), __dmul_rn((double)nj[a], (double)nj[a])));
    }
    return __dmul_rn(0.5 * m, __dsub_rn(e1, e0));
}

// Apply scatter events in ascending key order per particle.  One CTA; each
// round applies every pending event whose key is the smallest pending key at
// both of its particles (a topological order of the conflict graph, equal to
// sequential key order because events on disjoint particles commute).
template <class R>
__global__ void __launch_bounds__(1024) k_resolve(const sidm_event* __restrict__ ev, int64_t cap, R* vel, int64_t N,
                                                  const double* __restrict__ mass, unsigned long long* claim,
                                                  uint32_t* hits, uint8_t* done, DevCounters* cnt,
                                                  sidm_step_stats* st, int max_rounds, const float* sump, int use_sump)
{
    __shared__ unsigned int s_rem;
    __shared__ unsigned long long s_multi;
    const unsigned long long n_all = cnt->ev_count;
    if (threadIdx.x == 0) { s_multi = 0ull; s_rem = 0u; }
    __syncthreads();
    unsigned int status = 0u;
    unsigned int rounds = 0u;
    if (n_all > (unsigned long long)cap) {
        status |= SIDM_DEV_EVENT_OVERFLOW;
    } else if (n_all > 0ull) {
        const int64_t n = (int64_t)n_all;
        unsigned long long multi = 0ull;
        for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
            done[e] = 0;
            if (atomicAdd(&hits[ev[e].i], 1u) == 1u) ++multi;
            if (atomicAdd(&hits[ev[e].j], 1u) == 1u) ++multi;
        }
        atomicAdd(&s_multi, multi);
        __syncthreads();
        while (true) {
            // phase A: claim the smallest pending key at each particle
            for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
                if (__ldcg(done + e)) continue;
                atomicMin(&claim[ev[e].i], ev[e].key);
                atomicMin(&claim[ev[e].j], ev[e].key);
            }
            __syncthreads();
            // phase B: apply events minimal at both particles
            for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
                if (__ldcg(done + e)) continue;
                const sidm_event E = ev[e];
                if (__ldcg(claim + E.i) != E.key || __ldcg(claim + E.j) != E.key) continue;
                fx_add(cnt, apply_isotropic<R>(E, vel, N, mass));
                done[e] = 1;
            }
            __syncthreads();
            // phase C: release claims of everything pending at the start of the round
            unsigned int rem = 0u;
            for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
                claim[ev[e].i] = ~0ull;
                claim[ev[e].j] = ~0ull;
                if (!__ldcg(done + e)) ++rem;
            }
            if (threadIdx.x == 0) s_rem = 0u;
            __syncthreads();
            if (rem) atomicAdd(&s_rem, rem);
            __syncthreads();
            ++rounds;
            const unsigned int remaining = s_rem;
            __syncthreads();
            if (remaining == 0u) break;
            if ((int)rounds >= max_rounds) { status |= SIDM_DEV_ROUNDS; break; }
        }
        for (int64_t e = threadIdx.x; e < n; e += blockDim.x) { hits[ev[e].i] = 0u; hits[ev[e].j] = 0u; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (status) raise_status(cnt, status);
        st->n_events = n_all;
        st->n_multi = s_multi;
        st->rounds = rounds;
        st->status = status;
        const unsigned long long hi = cnt->de_hi, lo = cnt->de_lo;
        st->d_energy = ldexp((double)(long long)hi, -16) + ldexp((double)lo, -80);
    }
    if (use_sump) {   // max_i sum_j P_ij
        float m = 0.f;
        for (int64_t s = threadIdx.x; s < N; s += blockDim.x) m = fmaxf(m, sump[s]);
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) atomicMax((unsigned int*)&st->max_sum_p, __float_as_uint(m));
    }
}

// ---- a4 for forward-dominated halos: per-particle interaction lists -------
// Every in-range pair of such a halo is a record, so a particle takes part in
// hundreds of them per step and key order needs thousands of rounds.  Each
// particle gets the list of its records sorted by partner id, which is
// ascending key order for that particle (records (c, a), c < a, precede the
// records (a, b), b > a).  A round applies every record that is the next
// pending record of both its particles -- exactly the rounds of the claims
// above -- but looks only at the head of each active particle.

// 128-bit fixed-point accumulator in registers (units of 2^-80), merged into
// the global one once per warp: integer sums commute, so the total does not
// depend on the order of the records.
struct Fx128 {
    unsigned long long lo = 0ull, hi = 0ull;
    __device__ void add(double v)
    {
        const double hi_d = floor(ldexp(v, 16));
        const double lo_d = ldexp(v, 80) - ldexp(hi_d, 64);
        const unsigned long long l = lo_d >= 18446744073709551615.0 ? 0xFFFFFFFFFFFFFFFFull : __double2ull_rz(lo_d);
        const unsigned long long h = (unsigned long long)(long long)hi_d;
        lo += l;
        hi += h + (lo < l ? 1ull : 0ull);
    }
};

// List entries of the records: entry 2e for particle i, 2e + 1 for particle j,
// key = particle index << 27 | partner id.
__global__ void k_list_keys(const sidm_event* __restrict__ ev, int64_t n, unsigned long long* __restrict__ key,
                            uint32_t* __restrict__ val)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const sidm_event E = ev[e];
        const unsigned long long a = (E.key >> 27) & (kIdLimit - 1u), b = E.key & (kIdLimit - 1u);
        key[2 * e] = ((unsigned long long)E.i << 27) | b;
        key[2 * e + 1] = ((unsigned long long)E.j << 27) | a;
        val[2 * e] = (uint32_t)e;
        val[2 * e + 1] = (uint32_t)e;
    }
}

// Runs of the sorted entries: start and length of each particle's list, the
// initial active list, and the number of particles in two or more records.
__global__ void k_list_runs(const unsigned long long* __restrict__ key, int64_t m, uint32_t* __restrict__ start,
                            uint32_t* __restrict__ len, uint32_t* __restrict__ act, uint32_t* __restrict__ lcnt)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < m; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = (uint32_t)(key[s] >> 27);
        if (s > 0 && (uint32_t)(key[s - 1] >> 27) == p) continue;
        int64_t e = s + 1;
        while (e < m && (uint32_t)(key[e] >> 27) == p) ++e;
        start[p] = (uint32_t)s;
        len[p] = (uint32_t)(e - s);
        act[atomicAdd(&lcnt[0], 1u)] = p;
        if (e - s > 1) atomicAdd(&lcnt[2], 1u);
    }
}

// Grid-wide barrier of a cooperative launch (every CTA resident): arrival
// count work[2], generation work[3].  The wait gives up after kBarrierNs of
// %globaltimer time and returns false in every thread of the CTA.
constexpr unsigned long long kBarrierNs = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ bool grid_barrier(DevCounters* cnt)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* gen = &cnt->work[3];
        int ok = 1;
        __threadfence();
        const unsigned int g = *gen;
        if (atomicAdd(&cnt->work[2], 1u) == gridDim.x - 1) {
            atomicExch(&cnt->work[2], 0u);
            __threadfence();
            atomicAdd(&cnt->work[3], 1u);
        } else {
            const unsigned long long t0 = now_ns();
            while (*gen == g) {
                if (now_ns() - t0 > kBarrierNs) { ok = 0; break; }
                __nanosleep(100);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

struct ListResolve {
    const sidm_event* ev;
    const double* evg;
    const sidm_xs* xs;
    const double* mass;
    const uint32_t* lval;     // sorted entries: record index per list slot
    const uint32_t* start;
    const uint32_t* len;
    uint32_t* ptr;            // next pending entry of each list (zero at rest)
    uint32_t* act;            // [2][N] active particles (ping-pong)
    uint32_t* lcnt;           // [0], [1]: active counts; [2] multi-hit; [3] rounds; [4] status
    uint8_t* done;            // [records], zero at entry
    void* vel;
    int64_t N;
    int64_t n_rec;
    DevCounters* cnt;
};

template <class R>
__global__ void __launch_bounds__(256) k_resolve_lists(ListResolve q)
{
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    R* vel = (R*)q.vel;
    Fx128 acc;
    int cur = 0;
    unsigned int rounds = 0u, status = 0u;
    unsigned int n_cur = *(volatile unsigned int*)&q.lcnt[0];
    while (n_cur > 0u) {
        const uint32_t* act = q.act + (size_t)cur * q.N;
        uint32_t* nxt = q.act + (size_t)(cur ^ 1) * q.N;
        if (tid == 0) q.lcnt[cur ^ 1] = 0u;
        // apply every record that heads both of its particles' lists (by the
        // particle of lower index); the applied records touch disjoint particles
        for (int64_t a = tid; a < n_cur; a += T) {
            const uint32_t p = act[a];
            const uint32_t e = q.lval[q.start[p] + __ldcg(q.ptr + p)];
            const sidm_event E = q.ev[e];
            const uint32_t o = E.i == p ? E.j : E.i;
            if (p > o || q.lval[q.start[o] + __ldcg(q.ptr + o)] != e) continue;
            const sidm_xs xs = q.xs[(int)(E.key >> 54)];
            acc.add(xs.angular ? apply_drag<R>(E, q.evg[e], xs, vel, q.N, q.mass) : apply_isotropic<R>(E, vel, q.N, q.mass));
            __stcg(q.done + e, (uint8_t)1);
        }
        if (!grid_barrier(q.cnt)) { status |= SIDM_DEV_WAIT_TIMEOUT; break; }
        // advance the lists whose head was applied; keep the unfinished ones
        for (int64_t a = tid; a < n_cur; a += T) {
            const uint32_t p = act[a];
            uint32_t k = __ldcg(q.ptr + p);
            if (__ldcg(q.done + q.lval[q.start[p] + k])) __stcg(q.ptr + p, ++k);
            if (k < q.len[p]) nxt[atomicAdd(&q.lcnt[cur ^ 1], 1u)] = p;
        }
        ++rounds;
        if (!grid_barrier(q.cnt)) { status |= SIDM_DEV_WAIT_TIMEOUT; break; }
        n_cur = *(volatile unsigned int*)&q.lcnt[cur ^ 1];
        cur ^= 1;
        if ((int64_t)rounds > q.n_rec) { status |= SIDM_DEV_ROUNDS; break; }   // cannot happen: >= 1 record per round
    }
    // the pair energy changes: warp sums of the 128-bit accumulators, one
    // global addition per warp
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long l = __shfl_xor_sync(0xffffffffu, acc.lo, o);
        const unsigned long long h = __shfl_xor_sync(0xffffffffu, acc.hi, o);
        acc.lo += l;
        acc.hi += h + (acc.lo < l ? 1ull : 0ull);
    }
    if ((threadIdx.x & 31) == 0 && (acc.lo | acc.hi)) {
        const unsigned long long old = atomicAdd(&q.cnt->de_lo, acc.lo);
        atomicAdd(&q.cnt->de_hi, acc.hi + (old + acc.lo < old ? 1ull : 0ull));
    }
    if (tid == 0) { q.lcnt[3] = rounds; if (status) atomicOr(&q.lcnt[4], status); }
    else if (status && threadIdx.x == 0) atomicOr(&q.lcnt[4], status);
}

// The lists' pointers back to zero (entries of the sorted lists).
__global__ void k_list_reset(const unsigned long long* __restrict__ key, int64_t m, uint32_t* __restrict__ ptr)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < m; s += (int64_t)gridDim.x * blockDim.x)
        ptr[(uint32_t)(key[s] >> 27)] = 0u;
}

// Step statistics of a list resolve (one thread).
__global__ void k_list_stats(int64_t n_rec, const uint32_t* __restrict__ lcnt, DevCounters* cnt, sidm_step_stats* st)
{
    const unsigned int status = lcnt[4];
    if (status) raise_status(cnt, status);
    st->n_events = (unsigned long long)n_rec;
    st->n_multi = lcnt[2];
    st->rounds = lcnt[3];
    st->status = status;
    const unsigned long long hi = cnt->de_hi, lo = cnt->de_lo;
    st->d_energy = ldexp((double)(long long)hi, -16) + ldexp((double)lo, -80);
}

__global__ void k_list_overflow(DevCounters* cnt, sidm_step_stats* st)
{
    raise_status(cnt, SIDM_DEV_EVENT_OVERFLOW);
    st->n_events = cnt->ev_count;
    st->status = SIDM_DEV_EVENT_OVERFLOW;
}

// ------------------------------------------------------------------ a5 reduce
// Per chunk of kChunk particles: the unscaled sums (|v|^2, vx, vy, vz) as
// double-doubles, exact integers for FP32 velocities (sidm_sum.cuh).
static_assert(kChunk <= sidm_sum::kMaxChunk, "chunk larger than the exact-sum windows allow");

template <class R>
__global__ void __launch_bounds__(sidm_sum::chunk_threads<R>()) k_energy_partial(const R* __restrict__ vel, int64_t N,
                                                                      const int32_t* __restrict__ chunk_halo,
                                                                      const int64_t* __restrict__ chunk_begin,
                                                                      const int64_t* __restrict__ halo_off,
                                                                      double* __restrict__ part)
{
    const int c = blockIdx.x;
    const int h = chunk_halo[c];
    const int64_t b = chunk_begin[c];
    int64_t e = b + kChunk;
    if (e > halo_off[h + 1]) e = halo_off[h + 1];
    sidm_sum::chunk_sums(vel, N, b, e, part + 8 * (int64_t)c);
}

// First merge level: one warp per group of up to kGroupChunks consecutive
// chunks of a halo (groups numbered halo by halo).
__global__ void k_energy_group(int H, int ngroup, const int32_t* __restrict__ group_off,
                               const int32_t* __restrict__ chunk_off, const double* __restrict__ part,
                               double* __restrict__ gpart)
{
    const int g = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (g >= ngroup) return;                             // whole warps
    int lo = 0, hi = H;                                  // the last halo h with group_off[h] <= g
    while (hi - lo > 1) { const int mid = (lo + hi) >> 1; if (group_off[mid] <= g) lo = mid; else hi = mid; }
    const int c0 = chunk_off[lo] + (g - group_off[lo]) * sidm_sum::kGroupChunks;
    const int c1 = min(c0 + sidm_sum::kGroupChunks, chunk_off[lo + 1]);
    sidm_sum::group_sums(part, c0, c1, gpart + 8 * (int64_t)g);
}

// Second level: one warp per halo over its groups, scaled by the particle mass.
__global__ void k_energy_final(int H, const int32_t* __restrict__ group_off, const double* __restrict__ mass,
                               const double* __restrict__ gpart, double* __restrict__ out, double* __restrict__ comp)
{
    const int h = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (h >= H) return;                                  // whole warps
    sidm_sum::halo_result(gpart, group_off[h], group_off[h + 1], mass[h], out + 4 * h, comp ? comp + 4 * h : nullptr);
}

// ------------------------------------------------------------------ harness
template <class R>
__global__ void k_drift(int64_t N, int H, const int64_t* __restrict__ halo_off, const double* __restrict__ dt,
                        double* __restrict__ pos, const R* __restrict__ vel)
{
    // two particles per thread and trip, their loads issued together
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s0 < N; s0 += 2 * stride) {
        double x[2][3];
        R v[2][3];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t s = s0 + u * stride;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                x[u][a] = s < N ? pos[a * N + s] : 0.0;
                v[u][a] = s < N ? vel[a * N + s] : R(0);
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t s = s0 + u * stride;
            if (s >= N) break;
            const double d = dt[H == 1 ? 0 : halo_of(halo_off, H, s)];
#pragma unroll
            for (int a = 0; a < 3; ++a) pos[a * N + s] = __fma_rn((double)v[u][a], d, x[u][a]);   // one FP64 op
        }
    }
}

// Reflecting sphere per halo: an outward-moving particle outside it gets the
// radial part of its velocity reversed (speed kept).
template <class R>
__global__ void k_reflect(int64_t N, int H, const int64_t* __restrict__ halo_off, const double* __restrict__ bound,
                          const double* __restrict__ pos, R* __restrict__ vel)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
        const double* b = bound + 4 * halo_of(halo_off, H, s);
        const double rb = b[3];
        if (!(rb > 0.0)) continue;
        const double dx = pos[s] - b[0], dy = pos[N + s] - b[1], dz = pos[2 * N + s] - b[2];
        const double d2 = dx * dx + dy * dy + dz * dz;
        if (!(d2 > rb * rb)) continue;
        const double vx = vel[s], vy = vel[N + s], vz = vel[2 * N + s];
        const double vr = vx * dx + vy * dy + vz * dz;
        if (!(vr > 0.0)) continue;
        const double k = 2.0 * vr / d2;
        vel[s] = (R)(vx - k * dx);
        vel[N + s] = (R)(vy - k * dy);
        vel[2 * N + s] = (R)(vz - k * dz);
    }
}

template <class R>
__global__ void k_lambda_eval(int64_t n, const double* __restrict__ d, const double* __restrict__ hi,
                              const double* __restrict__ hj, double* __restrict__ out, const R* __restrict__ T)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = (double)lambda_lookup<R>(T, (R)d[t], (R)hi[t], (R)hj[t]);
}

// ------------------------------------------------------------------ Lambda table (host)
// Gauss-Legendre nodes on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) { double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-17) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) { double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Cubic spline of unit support and its first radial moment in closed form:
// S(t) = int_0^t t' W_1(t') dt'.
double spline_w1(double t)
{
    if (t < 0.0 || t >= 1.0) return 0.0;
    const double c = 8.0 / M_PI;
    if (t < 0.5) return c * (1.0 - 6.0 * t * t + 6.0 * t * t * t);
    const double u = 1.0 - t;
    return c * 2.0 * u * u * u;
}

double spline_s1(double t)
{
    const double c = 8.0 / M_PI;
    auto inner = [&](double q) { return c * (0.5 * q * q - 1.5 * q * q * q * q + 1.2 * q * q * q * q * q); };
    auto outer = [&](double q) { double u = 1.0 - q; return -2.0 * c * (0.25 * u * u * u * u - 0.2 * u * u * u * u * u); };
    if (t <= 0.0) return 0.0;
    if (t < 0.5) return inner(t);
    const double q = t < 1.0 ? t : 1.0;
    return inner(0.5) + outer(q) - outer(0.5);
}

// Lambda(d; a, b) for kernels of support a (at the origin) and b (at distance d):
//   (2 pi / d) int r W_a(r) [S_b(r + d) - S_b(|r - d|)] dr, S_b(s) = S_1(s/b)/b,
// piecewise Gauss-Legendre between the breakpoints of the polynomial pieces.
double lambda_host(double d, double a, double b, const double* gx, const double* gw, int ng)
{
    if (d >= a + b) return 0.0;
    auto Sb = [&](double s) { return spline_s1(s / b) / b; };
    auto Wa = [&](double r) { return spline_w1(r / a) / (a * a * a); };
    auto Wb = [&](double r) { return spline_w1(r / b) / (b * b * b); };
    std::vector<double> br;
    if (d == 0.0) {
        const double top = std::min(a, b);
        br = {0.0, top};
        for (double v : {0.5 * a, 0.5 * b}) if (v > 0.0 && v < top) br.push_back(v);
        std::sort(br.begin(), br.end());
        double acc = 0.0;
        for (size_t p = 0; p + 1 < br.size(); ++p) {
            const double m = 0.5 * (br[p] + br[p + 1]), hw = 0.5 * (br[p + 1] - br[p]);
            for (int g = 0; g < ng; ++g) { const double r = m + hw * gx[g]; acc += gw[g] * hw * r * r * Wa(r) * Wb(r); }
        }
        return 4.0 * M_PI * acc;
    }
    const double lo = std::max(0.0, d - b), hi = std::min(a, d + b);
    if (hi <= lo) return 0.0;
    br = {lo, hi};
    for (double v : {0.5 * a, a, d, d - 0.5 * b, d + 0.5 * b, d - b, d + b, 0.5 * b - d, b - d})
        if (v > lo && v < hi) br.push_back(v);
    std::sort(br.begin(), br.end());
    double acc = 0.0;
    for (size_t p = 0; p + 1 < br.size(); ++p) {
        const double m = 0.5 * (br[p] + br[p + 1]), hw = 0.5 * (br[p + 1] - br[p]);
        if (hw <= 0.0) continue;
        for (int g = 0; g < ng; ++g) {
            const double r = m + hw * gx[g];
            acc += gw[g] * hw * r * Wa(r) * (Sb(r + d) - Sb(std::fabs(r - d)));
        }
    }
    return 2.0 * M_PI * acc / d;
}

void lambda_table(std::vector<double>& T)
{
    const int ng = 10;
    double gx[16], gw[16];
    gauss_legendre(ng, gx, gw);
    T.assign((size_t)kLamNR * kLamNX, 0.0);
    for (int r = 0; r < kLamNR; ++r) {
        const double rho = (double)r / (kLamNR - 1);
        for (int c = 0; c < kLamNX; ++c) {
            const double x = (double)c / (kLamNX - 1);
            T[(size_t)r * kLamNX + c] = rho == 0.0 ? spline_w1(x) : lambda_host(x * (1.0 + rho), 1.0, rho, gx, gw, ng);
        }
    }
}

template <class T>
cudaError_t dev_alloc(T** p, size_t count)
{
    return cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
}

int grid_for(sidm_ctx* c, int64_t n, int threads)
{
    int64_t g = cdiv(n, threads);
    int64_t cap = (int64_t)c->sm_count * 8;
    return (int)std::max<int64_t>(1, std::min(g, cap));
}

}  // namespace

// ======================================================================= host
namespace sidm {

int set_err(sidm_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg;
    return code;
}

int cuda_check(sidm_ctx* c, cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return SIDM_OK;
    return set_err(c, SIDM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

cudaError_t ensure_device(sidm_ctx* c)
{
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return e;
    return cur == c->dev ? cudaSuccess : cudaSetDevice(c->dev);
}

// A kernel's dynamic shared-memory limit belongs to the kernel (per device),
// not to a context, so it is tracked process-wide and only ever raised: a
// launch of any context may use every size queried before, by any context.
static cudaError_t raise_smem_limit(const void* fn, size_t smem)
{
    struct Limit { int dev; const void* fn; size_t smem; };
    static std::mutex mu;
    static std::vector<Limit> limits;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    for (auto& l : limits)
        if (l.dev == dev && l.fn == fn) {
            if (smem <= l.smem) return cudaSuccess;
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) l.smem = smem;
            return e;
        }
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) limits.push_back({dev, fn, smem});
    return e;
}

int occupancy(sidm_ctx* c, const void* fn, int threads, size_t smem, int* occ)
{
    for (const auto& e : c->launch_cache)
        if (e.fn == fn && e.smem == smem) { *occ = e.occ; return SIDM_OK; }
    cudaError_t e = raise_smem_limit(fn, smem);
    if (e != cudaSuccess) return cuda_check(c, e, "shared-memory attribute");
    int o = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, threads, smem);
    if (e != cudaSuccess) return cuda_check(c, e, "occupancy");
    c->launch_cache.push_back({fn, smem, o});
    *occ = o;
    return SIDM_OK;
}

int timer_begin(sidm_ctx* c, int slot, cudaStream_t s)
{
    if (!(c->cfg.flags & SIDM_FLAG_TIMING) || c->t_used >= kTimerCap) return -1;
    const int idx = c->t_used++;
    c->t_slot[idx] = (int8_t)slot;
    cudaEventRecord(c->t_ev[2 * idx], s);
    return idx;
}

void timer_end(sidm_ctx* c, int idx, cudaStream_t s)
{
    if (idx >= 0) cudaEventRecord(c->t_ev[2 * idx + 1], s);
}

}  // namespace sidm

#define SIDM_LAUNCH(c, ...)                                                     \
    do {                                                                        \
        __VA_ARGS__;                                                            \
        (c)->launches++;                                                        \
        cudaError_t _e = cudaGetLastError();                                    \
        if (_e != cudaSuccess) return cuda_check((c), _e, "kernel launch");     \
    } while (0)

#define SIDM_CUDA(c, call)                                                      \
    do {                                                                        \
        cudaError_t _e = (call);                                                \
        if (_e != cudaSuccess) return cuda_check((c), _e, #call);               \
    } while (0)

// Stable LSD radix sort of (ka, va)[0, n) by the low 8 * passes key bits,
// ping-ponging with (kb, vb); on return ka/va hold the sorted pairs.
// With counted, the digit counts of every pass are already in d_sort_hist
// (taken by the kernel that made the keys, after sort_prepare).
static int sort_prepare(sidm_ctx* c, cudaStream_t s)
{
    SIDM_CUDA(c, cudaMemsetAsync(c->d_sort_hist, 0, sizeof(uint32_t) * sidm_sort::kMaxPasses * 257, s));
    return SIDM_OK;
}

static int radix_sort(sidm_ctx* c, unsigned long long*& ka, uint32_t*& va, unsigned long long*& kb, uint32_t*& vb,
                      int64_t n, int passes, cudaStream_t s, bool counted = false)
{
    using namespace sidm_sort;
    if (n <= 0) return SIDM_OK;
    const int64_t tiles = cdiv(n, kTile);
    if (tiles > c->sort_tiles_cap || passes < 1 || passes > kMaxPasses || n >= ((int64_t)1 << 32))
        return set_err(c, SIDM_ECAPACITY, "radix sort scratch too small");
    uint32_t* hist = c->d_sort_hist;
    uint32_t* tickets = hist + kMaxPasses * 256;
    if (!counted) {
        if (int rc = sort_prepare(c, s)) return rc;
        const int cgrid = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, kThreads * 4), (int64_t)c->sm_count * 4));
        SIDM_LAUNCH(c, k_sort_count<<<cgrid, kThreads, 0, s>>>(ka, n, passes, hist));
    }
    // persistent CTAs, as many as fit on the GPU at once
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, (int64_t)c->sm_count * kPassCtas);
    for (int p = 0; p < passes; ++p) {
        SIDM_CUDA(c, cudaMemsetAsync(c->d_sort_status, 0, sizeof(unsigned long long) * 256 * (size_t)tiles, s));
        const bool bulk = ((reinterpret_cast<uintptr_t>(ka) | reinterpret_cast<uintptr_t>(va)) & 15u) == 0u;
        SIDM_LAUNCH(c, k_sort_pass<<<grid, kThreads, kSmemBytes, s>>>(
            ka, va, n, 8 * p, (int)tiles, bulk, hist + 256 * p, c->d_sort_status, tickets + p, kb, vb,
            &c->d_cnt->status, SIDM_DEV_WAIT_TIMEOUT));
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    return SIDM_OK;
}

static void free_all(sidm_ctx* c)
{
    void* ptrs[] = {c->d_halo_off, c->d_halo_pad, c->d_leaf_off, c->d_lvl_off, c->d_top, c->d_ngb, c->d_leaf_halo, c->d_knn_redo,
                    c->d_chunk_halo, c->d_chunk_begin, c->d_frame, c->d_key, c->d_key2, c->d_val, c->d_val2,
                    c->d_sort_status, c->d_sort_hist, c->d_P4, c->d_V4, c->d_ID, c->d_cell, c->d_cellb, c->d_nlo, c->d_nhi, c->d_perm, c->d_tmp_pos,
                    c->d_tmp_vel, c->d_tmp_id, c->d_claim, c->d_hits, c->d_done, c->d_ev, c->d_sump,
                    c->d_stats_own, c->d_cnt, c->d_epart, c->d_chunk_off, c->d_group_off, c->d_gpart, c->d_lam, c->d_hprev, c->d_dacc, c->d_halo_ord,
                    c->d_evg, c->d_lkey, c->d_lval, c->d_lstart, c->d_llen, c->d_lptr, c->d_lact,
                    c->d_lcnt};
    for (void* p : ptrs) if (p) cudaFree(p);
    if (c->d_stage) cudaFreeHost(c->d_stage);
    for (cudaEvent_t e : c->t_ev) if (e) cudaEventDestroy(e);
    c->t_ev.clear();
}

extern "C" const char* sidm_create_error(void) { return g_create_err.c_str(); }

extern "C" const char* sidm_last_error(const sidm_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : "null context";
}

extern "C" int64_t sidm_launch_count(const sidm_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" int sidm_create(sidm_ctx** out, const sidm_config* cfg)
{
    if (!out || !cfg) { g_create_err = "null argument"; return SIDM_EINVAL; }
    *out = nullptr;
    if (cfg->n_max < 1 || cfg->n_max >= (1ll << 31)) { g_create_err = "n_max must be in [1, 2^31)"; return SIDM_EINVAL; }
    if (cfg->halo_max < 1 || cfg->halo_max > kMaxHalos) { g_create_err = "halo_max must be in [1, 1024]"; return SIDM_EINVAL; }
    if (cfg->ngb_max < 1 || cfg->ngb_max > kMaxNgb) { g_create_err = "ngb_max must be in [1, 128]"; return SIDM_EINVAL; }
    if (cfg->event_cap < 1) { g_create_err = "event_cap must be >= 1"; return SIDM_EINVAL; }
    if ((cfg->flags & SIDM_FLAG_DRAG) && cfg->event_cap >= (1ll << 31)) {
        g_create_err = "event_cap must be below 2^31 with SIDM_FLAG_DRAG"; return SIDM_EINVAL;
    }
    if (cfg->precision != SIDM_MIXED && cfg->precision != SIDM_FP64) { g_create_err = "bad precision"; return SIDM_EINVAL; }
    if (cfg->knn_warps < 0 || cfg->knn_warps > 16) { g_create_err = "knn_warps must be in [0, 16]"; return SIDM_EINVAL; }
    if (cfg->pair_warps < 0 || cfg->pair_warps > 8) {       // the pair kernel is built for CTAs of <= 256 threads
        g_create_err = "pair_warps must be in [0, 8]"; return SIDM_EINVAL;
    }
    if (!(cfg->knn_groups == 0 || cfg->knn_groups == 2 || cfg->knn_groups == 4 || cfg->knn_groups == 8) ||
        !(cfg->knn_chains == 0 || cfg->knn_chains == 4 || cfg->knn_chains == 8) || cfg->knn_flush < 0 ||
        cfg->knn_flush > 32 || !(cfg->knn_slack == 0.f || (cfg->knn_slack >= 1.f && cfg->knn_slack <= 2.f)) ||
        cfg->pair_per_round < 0 || cfg->pair_per_round > 4 || cfg->knn_batch < 0 || cfg->knn_batch > 3 ||
        (cfg->knn_chains == 8 && cfg->knn_groups != 4)) {
        g_create_err = "launch knobs out of range (knn_groups 2/4/8, knn_chains 4/8 (8 with 4 groups), "
                       "knn_flush <= 32, knn_slack in [1, 2], pair_per_round <= 4, knn_batch <= 3)";
        return SIDM_EINVAL;
    }
    sidm_ctx* c = new sidm_ctx();
    c->cfg = *cfg;
    if (c->cfg.max_rounds <= 0) c->cfg.max_rounds = 256;
    c->knn_warps = cfg->knn_warps ? cfg->knn_warps : 8;
    c->pair_warps = cfg->pair_warps ? cfg->pair_warps : 8;
    auto fail = [&](const std::string& m, cudaError_t e) {
        g_create_err = m + ": " + cudaGetErrorString(e);
        free_all(c);
        delete c;
        return SIDM_ECUDA;
    };
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e != cudaSuccess) return fail("cudaSetDevice", e);
    c->dev = cfg->device;
    e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->dev);
    if (e != cudaSuccess) return fail("cudaDeviceGetAttribute", e);
    e = cudaFuncSetAttribute(sidm_sort::k_sort_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sidm_sort::kSmemBytes);
    if (e != cudaSuccess) return fail("cudaFuncSetAttribute k_sort_pass", e);

    const int64_t N = cfg->n_max, H = cfg->halo_max;
    const int64_t Lmax = N / kLeaf + H + 1;
    const int64_t Npad = Lmax * kLeaf;
    const bool fp64 = cfg->precision == SIDM_FP64;
    const size_t rs = fp64 ? 8 : 4;
    c->node_cap = 2 * Lmax + (int64_t)kMaxLevels * (H + 1);
    c->chunk_cap = N / kChunk + H + 1;
    // radix sort scratch: the cell build sorts N keys, the list resolve 2 event_cap
    c->sort_tiles_cap = cdiv((cfg->flags & SIDM_FLAG_DRAG) ? std::max<int64_t>(N, 2 * cfg->event_cap) : N,
                             sidm_sort::kTile);
    c->stage_bytes = sizeof(int64_t) * (size_t)(8 * (H + 1) + kMaxLevels * (H + 1) + 2 * c->chunk_cap + 64);
#define ALLOC(p, n) do { e = dev_alloc(&(p), (size_t)(n)); if (e != cudaSuccess) return fail("cudaMalloc " #p, e); } while (0)
    ALLOC(c->d_halo_off, H + 1);
    ALLOC(c->d_halo_pad, H + 1);
    ALLOC(c->d_leaf_off, H + 1);
    ALLOC(c->d_lvl_off, kMaxLevels * (H + 1));
    ALLOC(c->d_top, H);
    ALLOC(c->d_ngb, H);
    ALLOC(c->d_leaf_halo, Lmax);
    ALLOC(c->d_knn_redo, Lmax);
    ALLOC(c->d_chunk_halo, c->chunk_cap);
    ALLOC(c->d_chunk_begin, c->chunk_cap);
    ALLOC(c->d_frame, H);
    ALLOC(c->d_key, N);
    ALLOC(c->d_key2, N);
    ALLOC(c->d_val, N);
    ALLOC(c->d_val2, N);
    ALLOC(c->d_sort_status, 256 * c->sort_tiles_cap);
    ALLOC(c->d_sort_hist, sidm_sort::kMaxPasses * 257);
    e = cudaMalloc(&c->d_P4, (size_t)Npad * 4 * rs); if (e != cudaSuccess) return fail("cudaMalloc P4", e);
    e = cudaMalloc(&c->d_V4, (size_t)Npad * 4 * rs); if (e != cudaSuccess) return fail("cudaMalloc V4", e);
    ALLOC(c->d_ID, Npad);
    ALLOC(c->d_cell, Lmax);
    ALLOC(c->d_cellb, Lmax);
    ALLOC(c->d_nlo, c->node_cap);
    ALLOC(c->d_nhi, c->node_cap);
    ALLOC(c->d_perm, N);
    e = cudaMalloc(&c->d_hprev, (size_t)N * rs); if (e != cudaSuccess) return fail("cudaMalloc hprev", e);
    ALLOC(c->d_tmp_pos, 3 * N);
    e = cudaMalloc(&c->d_tmp_vel, (size_t)3 * N * rs); if (e != cudaSuccess) return fail("cudaMalloc tmp_vel", e);
    ALLOC(c->d_tmp_id, N);
    ALLOC(c->d_claim, N);
    ALLOC(c->d_hits, N);
    ALLOC(c->d_done, cfg->event_cap);
    ALLOC(c->d_ev, cfg->event_cap);
    ALLOC(c->d_sump, (cfg->flags & SIDM_FLAG_SUM_P) ? N : 1);
    ALLOC(c->d_dacc, (cfg->flags & SIDM_FLAG_LOCAL_DIAG) ? 5 * N : 1);
    ALLOC(c->d_stats_own, 1);
    ALLOC(c->d_cnt, 1);
    ALLOC(c->d_epart, 8 * c->chunk_cap);
    ALLOC(c->d_chunk_off, H + 1);
    ALLOC(c->d_group_off, H + 1);
    ALLOC(c->d_gpart, 8 * (c->chunk_cap / sidm_sum::kGroupChunks + H + 1));
    ALLOC(c->d_halo_ord, H);
    if (cfg->flags & SIDM_FLAG_DRAG) {
        const int64_t m = 2 * cfg->event_cap;
        ALLOC(c->d_evg, cfg->event_cap);
        ALLOC(c->d_lkey, 2 * m);
        ALLOC(c->d_lval, 2 * m);
        ALLOC(c->d_lstart, N);
        ALLOC(c->d_llen, N);
        ALLOC(c->d_lptr, N);
        ALLOC(c->d_lact, 2 * N);
        ALLOC(c->d_lcnt, 8);
    }
#undef ALLOC
    e = cudaMallocHost((void**)&c->d_stage, c->stage_bytes);
    if (e != cudaSuccess) return fail("cudaMallocHost", e);
    // Lambda table: FP64 quadrature on the host, stored in the form's precision.
    std::vector<double> T;
    lambda_table(T);
    gauss_legendre(8, c->gl8x, c->gl8w);
    if (fp64) {
        e = cudaMalloc(&c->d_lam, T.size() * 8); if (e != cudaSuccess) return fail("cudaMalloc lam", e);
        e = cudaMemcpy(c->d_lam, T.data(), T.size() * 8, cudaMemcpyHostToDevice);
    } else {
        std::vector<float> Tf(T.begin(), T.end());
        e = cudaMalloc(&c->d_lam, Tf.size() * 4); if (e != cudaSuccess) return fail("cudaMalloc lam", e);
        e = cudaMemcpy(c->d_lam, Tf.data(), Tf.size() * 4, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return fail("cudaMemcpy lam", e);
    e = cudaMemset(c->d_hits, 0, sizeof(uint32_t) * (size_t)N); if (e != cudaSuccess) return fail("memset", e);
    e = cudaMemset(c->d_cnt, 0, sizeof(DevCounters)); if (e != cudaSuccess) return fail("memset", e);
    e = cudaMemset(c->d_claim, 0xFF, sizeof(unsigned long long) * (size_t)N); if (e != cudaSuccess) return fail("memset", e);
    if (c->d_lptr) { e = cudaMemset(c->d_lptr, 0, sizeof(uint32_t) * (size_t)N); if (e != cudaSuccess) return fail("memset", e); }
    if (cfg->flags & SIDM_FLAG_TIMING) {
        c->t_ev.assign(2 * kTimerCap, nullptr);
        c->t_slot.assign(kTimerCap, 0);
        for (auto& ev : c->t_ev) {
            e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return fail("cudaEventCreate", e);
        }
    }
    e = cudaDeviceSynchronize(); if (e != cudaSuccess) return fail("sync", e);
    *out = c;
    return SIDM_OK;
}

extern "C" int sidm_destroy(sidm_ctx* c)
{
    if (!c) return SIDM_OK;
    cudaSetDevice(c->dev);
    cudaDeviceSynchronize();
    free_all(c);
    delete c;
    return SIDM_OK;
}

// Host-side layout of a halo set (leaves, tree levels, reduction chunks).
static int make_layout(sidm_ctx* c, int H, const int64_t* off, LayoutHost& L)
{
    L = LayoutHost();
    L.H = H;
    L.halo_off.assign(off, off + H + 1);
    L.N = off[H];
    L.halo_pad.assign(H + 1, 0);
    L.leaf_off.assign(H + 1, 0);
    for (int h = 0; h < H; ++h) {
        const int64_t n = off[h + 1] - off[h];
        const int64_t nl = cdiv(n, kLeaf);
        L.halo_pad[h + 1] = L.halo_pad[h] + nl * kLeaf;
        L.leaf_off[h + 1] = L.leaf_off[h] + (int32_t)nl;
    }
    L.Npad = L.halo_pad[H];
    L.L = L.leaf_off[H];
    L.top.assign(H, 0);
    int maxtop = 0;
    for (int h = 0; h < H; ++h) {
        int64_t cnt = L.leaf_off[h + 1] - L.leaf_off[h];
        int t = 0;
        while (cnt > kArity) { cnt = cdiv(cnt, kArity); ++t; }
        L.top[h] = t;
        maxtop = std::max(maxtop, t);
    }
    L.nlev = maxtop + 1;
    if (L.nlev > kMaxLevels) return set_err(c, SIDM_ECAPACITY, "too many tree levels");
    L.lvl_off.assign((size_t)L.nlev * (H + 1), 0);
    int64_t base = 0;
    for (int l = 0; l < L.nlev; ++l) {
        int64_t run = base;
        for (int h = 0; h < H; ++h) {
            L.lvl_off[(size_t)l * (H + 1) + h] = (int32_t)run;
            int64_t cnt = L.leaf_off[h + 1] - L.leaf_off[h];
            for (int k = 0; k < l; ++k) cnt = cdiv(cnt, kArity);
            run += cnt;
        }
        L.lvl_off[(size_t)l * (H + 1) + H] = (int32_t)run;
        base = run;
    }
    if (base > c->node_cap) return set_err(c, SIDM_ECAPACITY, "tree node capacity exceeded");
    for (int h = 0; h < H; ++h)
        for (int64_t b = off[h]; b < off[h + 1]; b += kChunk) { L.chunk_halo.push_back(h); L.chunk_begin.push_back(b); }
    L.nchunk = (int)L.chunk_halo.size();
    L.chunk_off.assign(H + 1, 0);
    L.group_off.assign(H + 1, 0);
    for (int h = 0; h < H; ++h) {
        const int nc = (int)cdiv(off[h + 1] - off[h], kChunk);
        L.chunk_off[h + 1] = L.chunk_off[h] + nc;
        L.group_off[h + 1] = L.group_off[h] + (int)cdiv(nc, sidm_sum::kGroupChunks);
    }
    L.ngroup = L.group_off[H];
    if (L.nchunk > c->chunk_cap) return set_err(c, SIDM_ECAPACITY, "chunk capacity exceeded");
    int hb = 0;
    while ((1 << hb) < H) ++hb;
    L.sort_passes = (int)cdiv(kHaloShift + hb, 8);
    return SIDM_OK;
}

static int upload_layout(sidm_ctx* c, cudaStream_t s)
{
    const LayoutHost& L = c->lay;
    const int H = L.H;
    int64_t* st = c->d_stage;
    size_t o = 0;
    auto put = [&](const void* src, size_t bytes, void* dst) -> int {
        if ((o * 8 + bytes) > c->stage_bytes) return set_err(c, SIDM_ECAPACITY, "staging buffer too small");
        std::memcpy((char*)st + o * 8, src, bytes);
        cudaError_t e = cudaMemcpyAsync(dst, (char*)st + o * 8, bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_check(c, e, "layout upload");
        o += (bytes + 7) / 8;
        return SIDM_OK;
    };
    int rc;
    if ((rc = put(L.halo_off.data(), 8 * (H + 1), c->d_halo_off))) return rc;
    if ((rc = put(L.halo_pad.data(), 8 * (H + 1), c->d_halo_pad))) return rc;
    if ((rc = put(L.leaf_off.data(), 4 * (H + 1), c->d_leaf_off))) return rc;
    if ((rc = put(L.lvl_off.data(), 4 * L.lvl_off.size(), c->d_lvl_off))) return rc;
    if ((rc = put(L.top.data(), 4 * H, c->d_top))) return rc;
    if ((rc = put(L.chunk_off.data(), 4 * (H + 1), c->d_chunk_off))) return rc;
    if ((rc = put(L.group_off.data(), 4 * (H + 1), c->d_group_off))) return rc;
    if (L.nchunk) {
        if ((rc = put(L.chunk_halo.data(), 4 * L.nchunk, c->d_chunk_halo))) return rc;
        if ((rc = put(L.chunk_begin.data(), 8 * L.nchunk, c->d_chunk_begin))) return rc;
    }
    SIDM_CUDA(c, cudaStreamSynchronize(s));   // staging buffer is reused
    return SIDM_OK;
}

template <class R>
static int build_impl(sidm_ctx* c, double* pos, R* vel, uint32_t* id, cudaStream_t s)
{
    const LayoutHost& L = c->lay;
    const int H = L.H;
    const int64_t N = L.N;
    if (N == 0) return SIDM_OK;
    // per-halo bounding box -> frame
    SIDM_CUDA(c, cudaMemsetAsync(c->d_cnt->bbox, 0xFF, sizeof(unsigned long long) * 3 * H, s));
    SIDM_CUDA(c, cudaMemsetAsync(c->d_cnt->bbox + 3 * H, 0x00, sizeof(unsigned long long) * 3 * H, s));
    SIDM_LAUNCH(c, k_bbox<<<L.nchunk * kBboxSplit, 256, 0, s>>>(pos, N, c->d_chunk_halo, c->d_chunk_begin, c->d_halo_off, H, c->d_cnt->bbox));
    SIDM_LAUNCH(c, k_frame<<<(H + 127) / 128, 128, 0, s>>>(H, c->d_halo_off, c->d_cnt->bbox, c->d_frame));
    if (int rc = sort_prepare(c, s)) return rc;
    SIDM_LAUNCH(c, k_keys<<<grid_for(c, N, 256), 256, 0, s>>>(pos, N, c->d_halo_off, H, c->d_frame, c->d_key, c->d_val,
                                                               L.sort_passes, c->d_sort_hist));
    // stable LSD radix sort
    unsigned long long *ka = c->d_key, *kb = c->d_key2;
    uint32_t *va = c->d_val, *vb = c->d_val2;
    if (int rc = radix_sort(c, ka, va, kb, vb, N, L.sort_passes, s, true)) return rc;
    // leaves, gather, copy back into the caller's arrays
    SIDM_LAUNCH(c, k_leaf_fill<<<(L.L + 255) / 256, 256, 0, s>>>(L.L, H, c->d_leaf_off, c->d_halo_off, ka, c->d_frame,
                                                                  c->d_leaf_halo, c->d_cell, c->d_cellb));
    const bool mixed = c->cfg.precision == SIDM_MIXED;
    using V = typename Vec4<R>::T;
    // the last kernel sizes, in the order the caller's arrays had after that
    // call, seed the next search (only a guess: the search stays exact)
    const R* hprev = (c->warm_enabled && c->hprev_valid) ? (const R*)c->d_hprev : nullptr;
    c->guess_in_p4 = hprev != nullptr;
    c->hprev_valid = false;
    if (mixed)
        SIDM_LAUNCH(c, (k_gather_leaves<R><<<(unsigned)cdiv((int64_t)L.L * 32, 256), 256, 0, s>>>(
            L.L, N, c->d_leaf_halo, c->d_leaf_off, c->d_halo_off, c->d_cell, c->d_cellb, va, pos, vel, id,
            c->d_tmp_pos, (R*)c->d_tmp_vel, c->d_tmp_id, c->d_perm, (V*)c->d_P4, c->d_ID, c->d_cnt, hprev,
            c->d_nlo, c->d_nhi)));
    else
        SIDM_LAUNCH(c, (k_gather<R><<<grid_for(c, N, 256), 256, 0, s>>>(
            N, H, c->d_halo_off, c->d_halo_pad, ka, va, pos, vel, id,
            c->d_tmp_pos, (R*)c->d_tmp_vel, c->d_tmp_id, c->d_perm, (V*)c->d_P4, c->d_ID, c->d_cnt, hprev)));
    SIDM_CUDA(c, cudaMemcpyAsync(pos, c->d_tmp_pos, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s));
    SIDM_CUDA(c, cudaMemcpyAsync(vel, c->d_tmp_vel, sizeof(R) * 3 * N, cudaMemcpyDeviceToDevice, s));
    SIDM_CUDA(c, cudaMemcpyAsync(id, c->d_tmp_id, sizeof(uint32_t) * N, cudaMemcpyDeviceToDevice, s));
    if (!mixed)
        SIDM_LAUNCH(c, k_leaf_bbox<<<(L.L * 32 + 255) / 256, 256, 0, s>>>(L.L, N, c->d_leaf_halo, c->d_leaf_off,
                                                                           c->d_halo_off, c->d_frame, pos, c->d_nlo,
                                                                           c->d_nhi));
    for (int l = 1; l < L.nlev; ++l) {
        const int cnt = L.lvl_off[(size_t)l * (H + 1) + H] - L.lvl_off[(size_t)l * (H + 1)];
        SIDM_LAUNCH(c, k_tree_level<<<std::max(1, (cnt * 32 + 255) / 256), 256, 0, s>>>(l, H, c->d_lvl_off, c->d_nlo, c->d_nhi));
    }
    return SIDM_OK;
}

extern "C" int sidm_build_cells(sidm_ctx* c, int32_t n_halos, const int64_t* halo_off, double* pos, void* vel,
                                uint32_t* id, cudaStream_t s)
{
    if (!c) return SIDM_EINVAL;
    if (n_halos < 1 || n_halos > c->cfg.halo_max || !halo_off) return set_err(c, SIDM_EINVAL, "bad halo count");
    if (halo_off[0] != 0) return set_err(c, SIDM_EINVAL, "halo_off[0] must be 0");
    for (int h = 0; h < n_halos; ++h)
        if (halo_off[h + 1] < halo_off[h]) return set_err(c, SIDM_EINVAL, "halo_off must be non-decreasing");
    if (halo_off[n_halos] > c->cfg.n_max) return set_err(c, SIDM_ECAPACITY, "more particles than n_max");
    if (halo_off[n_halos] > 0 && (!pos || !vel || !id)) return set_err(c, SIDM_EINVAL, "null particle array");
    SIDM_CUDA(c, ensure_device(c));
    const bool same = c->has_layout && c->lay.H == n_halos &&
                      std::equal(halo_off, halo_off + n_halos + 1, c->lay.halo_off.begin());
    if (!same) {
        LayoutHost L;
        int rc = make_layout(c, n_halos, halo_off, L);
        if (rc) return rc;
        c->lay = L;
        c->has_layout = true;
        c->built = c->sized = false;
        c->hprev_valid = false;
        if ((rc = upload_layout(c, s))) { c->has_layout = false; return rc; }
    }
    const int tb = timer_begin(c, 0, s);
    int rc = c->cfg.precision == SIDM_FP64 ? build_impl<double>(c, pos, (double*)vel, id, s)
                                           : build_impl<float>(c, pos, (float*)vel, id, s);
    timer_end(c, tb, s);
    if (rc) return rc;
    c->built = true;
    c->sized = false;
    return SIDM_OK;
}

extern "C" int sidm_kernel_sizes(sidm_ctx* c, const int32_t* n_ngb, void* h_dev, cudaStream_t s)
{
    if (!c) return SIDM_EINVAL;
    if (!c->built) return set_err(c, SIDM_EINVAL, "sidm_build_cells must come first");
    if (!n_ngb || (!h_dev && c->lay.N > 0)) return set_err(c, SIDM_EINVAL, "null argument");
    const LayoutHost& L = c->lay;
    int kmax = 0;
    for (int h = 0; h < L.H; ++h) {
        const int64_t n = L.halo_off[h + 1] - L.halo_off[h];
        if (n == 0) continue;
        if (n_ngb[h] < 1 || n_ngb[h] > c->cfg.ngb_max)
            return set_err(c, SIDM_EINVAL, "n_ngb out of [1, ngb_max] for halo " + std::to_string(h));
        if (n_ngb[h] >= n)
            return set_err(c, SIDM_EINVAL, "halo " + std::to_string(h) + " has no more than n_ngb particles");
        kmax = std::max(kmax, n_ngb[h]);
    }
    SIDM_CUDA(c, ensure_device(c));
    if (c->ngb_host.size() != (size_t)L.H || !std::equal(n_ngb, n_ngb + L.H, c->ngb_host.begin())) {
        std::memcpy(c->d_stage, n_ngb, sizeof(int32_t) * L.H);
        SIDM_CUDA(c, cudaMemcpyAsync(c->d_ngb, c->d_stage, sizeof(int32_t) * L.H, cudaMemcpyHostToDevice, s));
        SIDM_CUDA(c, cudaStreamSynchronize(s));
        c->ngb_host.assign(n_ngb, n_ngb + L.H);
    }
    c->kmax_cur = kmax;
    if (L.N == 0) { c->sized = true; return SIDM_OK; }
    const bool use_guess = c->guess_in_p4 && c->ngb_prev == c->ngb_host;
    c->guess_in_p4 = false;
    int rc = launch_knn(c, h_dev, nullptr, 0, use_guess, s);
    if (rc) return rc;
    c->hprev_valid = true;
    c->ngb_prev = c->ngb_host;
    if (c->cfg.precision == SIDM_FP64)
        SIDM_LAUNCH(c, k_leaf_hmax<double><<<(L.L * 32 + 255) / 256, 256, 0, s>>>(L.L, L.H, c->d_leaf_halo, c->d_leaf_off,
                                                                                 c->d_halo_off, (const double4_16a*)c->d_P4, c->d_nlo));
    else
        SIDM_LAUNCH(c, k_leaf_hmax<float><<<(L.L * 32 + 255) / 256, 256, 0, s>>>(L.L, L.H, c->d_leaf_halo, c->d_leaf_off,
                                                                               c->d_halo_off, (const float4*)c->d_P4, c->d_nlo));
    for (int l = 1; l < L.nlev; ++l) {
        const int cnt = L.lvl_off[(size_t)l * (L.H + 1) + L.H] - L.lvl_off[(size_t)l * (L.H + 1)];
        SIDM_LAUNCH(c, k_tree_level<<<std::max(1, (cnt * 32 + 255) / 256), 256, 0, s>>>(l, L.H, c->d_lvl_off, c->d_nlo, c->d_nhi));
    }
    c->sized = true;
    return SIDM_OK;
}

extern "C" int sidm_neighbours(sidm_ctx* c, const int32_t* n_ngb, int32_t k_stride, uint32_t* nbr, cudaStream_t s)
{
    if (!c) return SIDM_EINVAL;
    if (c->cfg.precision != SIDM_MIXED) return set_err(c, SIDM_EINVAL, "neighbour lists: mixed form only");
    if (!c->sized) return set_err(c, SIDM_EINVAL, "sidm_kernel_sizes must come first");
    if (!n_ngb || !nbr) return set_err(c, SIDM_EINVAL, "null argument");
    for (int h = 0; h < c->lay.H; ++h)
        if (c->lay.halo_off[h + 1] > c->lay.halo_off[h] && (n_ngb[h] != c->ngb_host[h] || n_ngb[h] > k_stride))
            return set_err(c, SIDM_EINVAL, "n_ngb must match the kernel-size pass and fit k_stride");
    SIDM_CUDA(c, ensure_device(c));
    return launch_knn(c, nullptr, nbr, k_stride, false, s);
}

__global__ void k_max_sump(int64_t N, const float* __restrict__ sump, sidm_step_stats* st)
{
    float m = 0.f;
    for (int64_t s = threadIdx.x; s < N; s += blockDim.x) m = fmaxf(m, sump[s]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax((unsigned int*)&st->max_sum_p, __float_as_uint(m));
}

// a4 through per-particle interaction lists (contexts with SIDM_FLAG_DRAG; any
// mix of isotropic and forward-dominated halos).  Synchronises the stream once,
// to size the list sort from the number of records.
template <class R>
static int resolve_lists(sidm_ctx* c, const sidm_xs* xs, const double* mass, R* vel, sidm_step_stats* st, int use_sump,
                         cudaStream_t s)
{
    const LayoutHost& L = c->lay;
    const int tr = timer_begin(c, 3, s);
    unsigned long long n = 0ull;
    SIDM_CUDA(c, cudaMemcpyAsync(c->d_stage, &c->d_cnt->ev_count, sizeof(n), cudaMemcpyDeviceToHost, s));
    SIDM_CUDA(c, cudaStreamSynchronize(s));
    std::memcpy(&n, c->d_stage, sizeof(n));
    SIDM_CUDA(c, cudaMemsetAsync(c->d_lcnt, 0, 8 * sizeof(uint32_t), s));
    if (n > (unsigned long long)c->cfg.event_cap) {
        SIDM_LAUNCH(c, k_list_overflow<<<1, 1, 0, s>>>(c->d_cnt, st));
        timer_end(c, tr, s);
        return SIDM_OK;
    }
    const int64_t m = 2 * (int64_t)n;
    unsigned long long *ka = c->d_lkey, *kb = c->d_lkey + m;
    uint32_t *va = c->d_lval, *vb = c->d_lval + m;
    if (n > 0) {
        SIDM_CUDA(c, cudaMemsetAsync(c->d_done, 0, (size_t)n, s));
        SIDM_LAUNCH(c, k_list_keys<<<grid_for(c, (int64_t)n, 256), 256, 0, s>>>(c->d_ev, (int64_t)n, ka, va));
        // stable LSD radix sort of the entries by (particle index, partner id)
        int ib = 1;
        while (ib < 31 && ((int64_t)1 << ib) < L.N) ++ib;
        const int passes = (int)cdiv(27 + ib, 8);
        if (int rc = radix_sort(c, ka, va, kb, vb, m, passes, s)) return rc;
        SIDM_LAUNCH(c, k_list_runs<<<grid_for(c, m, 256), 256, 0, s>>>(ka, m, c->d_lstart, c->d_llen, c->d_lact, c->d_lcnt));
        SIDM_CUDA(c, cudaMemsetAsync(&c->d_cnt->work[2], 0, sizeof(unsigned int), s));
        ListResolve q;
        q.ev = c->d_ev; q.evg = c->d_evg; q.xs = xs; q.mass = mass; q.lval = va; q.start = c->d_lstart;
        q.len = c->d_llen; q.ptr = c->d_lptr; q.act = c->d_lact; q.lcnt = c->d_lcnt; q.done = c->d_done;
        q.vel = vel; q.N = L.N; q.n_rec = (int64_t)n; q.cnt = c->d_cnt;
        auto kern = k_resolve_lists<R>;
        int occ = 0;
        int rc = occupancy(c, (const void*)kern, 256, 0, &occ);
        if (rc) return rc;
        if (occ < 1) return set_err(c, SIDM_ECAPACITY, "list resolve does not fit on an SM");
        const int grid = c->sm_count * occ;       // every CTA resident: the rounds use a grid barrier
        void* args[] = {&q};
        SIDM_CUDA(c, cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(256), args, 0, s));
        c->launches++;
        SIDM_LAUNCH(c, k_list_reset<<<grid_for(c, m, 256), 256, 0, s>>>(ka, m, c->d_lptr));
    }
    SIDM_LAUNCH(c, k_list_stats<<<1, 1, 0, s>>>((int64_t)n, c->d_lcnt, c->d_cnt, st));
    if (use_sump) SIDM_LAUNCH(c, k_max_sump<<<1, 1024, 0, s>>>(L.N, c->d_sump, st));
    timer_end(c, tr, s);
    return SIDM_OK;
}

static int scatter_impl(sidm_ctx* c, uint64_t seed, uint64_t step, const sidm_xs* xs, const double* dt,
                        const double* mass, void* vel, sidm_step_stats* stats, cudaStream_t s)
{
    SIDM_CUDA(c, ensure_device(c));
    const LayoutHost& L = c->lay;
    sidm_step_stats* st = stats ? stats : c->d_stats_own;
    SIDM_CUDA(c, cudaMemsetAsync(st, 0, sizeof(sidm_step_stats), s));
    SIDM_CUDA(c, cudaMemsetAsync(c->d_cnt, 0, offsetof(DevCounters, work), s));
    if (c->cfg.flags & SIDM_FLAG_SUM_P) SIDM_CUDA(c, cudaMemsetAsync(c->d_sump, 0, sizeof(float) * std::max<int64_t>(L.N, 1), s));
    c->stepped = true;
    if (L.N == 0) return SIDM_OK;
    const bool fp64 = c->cfg.precision == SIDM_FP64;
    if (fp64)
        SIDM_LAUNCH(c, k_vel_refresh<double><<<grid_for(c, L.N, 256), 256, 0, s>>>(L.N, L.H, c->d_halo_off, c->d_halo_pad,
                                                                                  (const double*)vel, c->d_ID, (double4_16a*)c->d_V4));
    else
        SIDM_LAUNCH(c, k_vel_refresh<float><<<grid_for(c, L.N, 256), 256, 0, s>>>(L.N, L.H, c->d_halo_off, c->d_halo_pad,
                                                                                (const float*)vel, c->d_ID, (float4*)c->d_V4));
    int rc = launch_pairs(c, seed, step, xs, dt, mass, st, s);
    if (rc) return rc;
    const int use_sump = (c->cfg.flags & SIDM_FLAG_SUM_P) ? 1 : 0;
    if (c->cfg.flags & SIDM_FLAG_DRAG)
        return fp64 ? resolve_lists<double>(c, xs, mass, (double*)vel, st, use_sump, s)
                    : resolve_lists<float>(c, xs, mass, (float*)vel, st, use_sump, s);
    const int tr = timer_begin(c, 3, s);
    if (fp64)
        SIDM_LAUNCH(c, k_resolve<double><<<1, 1024, 0, s>>>(c->d_ev, c->cfg.event_cap, (double*)vel, L.N, mass, c->d_claim,
                                                          c->d_hits, c->d_done, c->d_cnt, st, c->cfg.max_rounds, c->d_sump, use_sump));
    else
        SIDM_LAUNCH(c, k_resolve<float><<<1, 1024, 0, s>>>(c->d_ev, c->cfg.event_cap, (float*)vel, L.N, mass, c->d_claim,
                                                         c->d_hits, c->d_done, c->d_cnt, st, c->cfg.max_rounds, c->d_sump, use_sump));
    timer_end(c, tr, s);
    return SIDM_OK;
}

extern "C" int sidm_timestep_criterion(sidm_ctx* c, double tau, double dt_min, double dt_max, int32_t n_bins,
                                       const double* dt, double* dt_out, int32_t* bin_out, double* dt_halo_min,
                                       cudaStream_t s)
{
    if (!c) return SIDM_EINVAL;
    if (!(c->cfg.flags & SIDM_FLAG_SUM_P)) return set_err(c, SIDM_EINVAL, "context built without SIDM_FLAG_SUM_P");
    if (!c->stepped) return set_err(c, SIDM_EINVAL, "sidm_scatter_step must come first");
    if (!(tau > 0.0) || !(dt_min >= 0.0) || !(dt_max >= dt_min) || !(dt_max > 0.0))
        return set_err(c, SIDM_EINVAL, "need 0 < tau and 0 <= dt_min <= dt_max, dt_max > 0");
    if (n_bins < 1 || n_bins > 32) return set_err(c, SIDM_EINVAL, "n_bins must be in 1..32");
    if (!dt) return set_err(c, SIDM_EINVAL, "null dt");
    SIDM_CUDA(c, ensure_device(c));
    const LayoutHost& L = c->lay;
    unsigned long long* ord = c->d_halo_ord;
    if (dt_halo_min) SIDM_CUDA(c, cudaMemsetAsync(ord, 0xFF, sizeof(unsigned long long) * L.H, s));
    if (L.N > 0)
        SIDM_LAUNCH(c, k_timestep<<<grid_for(c, L.N, 256), 256, 0, s>>>(L.N, L.H, c->d_halo_off, c->d_sump, dt, tau, dt_min,
                                                                      dt_max, n_bins, dt_out, bin_out,
                                                                      dt_halo_min ? ord : nullptr));
    if (dt_halo_min)
        SIDM_LAUNCH(c, k_halo_min_final<<<(L.H + 127) / 128, 128, 0, s>>>(L.H, ord, dt_max, dt_halo_min));
    return SIDM_OK;
}

extern "C" int sidm_local_diagnostics(sidm_ctx* c, const sidm_xs* xs, const double* mass, const void* vel, double G,
                                      void* out, cudaStream_t s)
{
    if (!c) return SIDM_EINVAL;
    if (!(c->cfg.flags & SIDM_FLAG_LOCAL_DIAG)) return set_err(c, SIDM_EINVAL, "context built without SIDM_FLAG_LOCAL_DIAG");
    if (!c->sized) return set_err(c, SIDM_EINVAL, "sidm_kernel_sizes must come first");
    if (!xs || !mass || ((!vel || !out) && c->lay.N > 0)) return set_err(c, SIDM_EINVAL, "null argument");
    if (!(G > 0.0)) return set_err(c, SIDM_EINVAL, "G must be positive");
    SIDM_CUDA(c, ensure_device(c));
    const LayoutHost& L = c->lay;
    if (L.N == 0) return SIDM_OK;
    const bool fp64 = c->cfg.precision == SIDM_FP64;
    SIDM_CUDA(c, cudaMemsetAsync(c->d_dacc, 0, sizeof(double) * 5 * L.N, s));
    if (fp64)
        SIDM_LAUNCH(c, k_vel_refresh<double><<<grid_for(c, L.N, 256), 256, 0, s>>>(L.N, L.H, c->d_halo_off, c->d_halo_pad,
                                                                                  (const double*)vel, c->d_ID, (double4_16a*)c->d_V4));
    else
        SIDM_LAUNCH(c, k_vel_refresh<float><<<grid_for(c, L.N, 256), 256, 0, s>>>(L.N, L.H, c->d_halo_off, c->d_halo_pad,
                                                                                (const float*)vel, c->d_ID, (float4*)c->d_V4));
    int rc = launch_pairs_diag(c, xs, mass, s);
    if (rc) return rc;
    const int blocks = (int)(((int64_t)L.L * kLeaf + 255) / 256);
    if (fp64)
        SIDM_LAUNCH(c, k_diag_final<double><<<blocks, 256, 0, s>>>(L.L, c->d_leaf_halo, c->d_leaf_off, c->d_halo_off,
                                                                   (const double4_16a*)c->d_P4, (const double4_16a*)c->d_V4,
                                                                   c->d_dacc, L.N, mass, xs, c->d_ngb, G, (double*)out));
    else
        SIDM_LAUNCH(c, k_diag_final<float><<<blocks, 256, 0, s>>>(L.L, c->d_leaf_halo, c->d_leaf_off, c->d_halo_off,
                                                                  (const float4*)c->d_P4, (const float4*)c->d_V4,
                                                                  c->d_dacc, L.N, mass, xs, c->d_ngb, G, (float*)out));
    return SIDM_OK;
}

extern "C" int sidm_scatter_step(sidm_ctx* c, uint64_t seed, uint64_t step, const sidm_xs* xs, const double* dt,
                                 const double* mass, void* vel, sidm_step_stats* stats, cudaStream_t s)
{
    if (!c) return SIDM_EINVAL;
    if (!c->sized) return set_err(c, SIDM_EINVAL, "sidm_kernel_sizes must come first");
    if (!xs || !dt || !mass || (!vel && c->lay.N > 0)) return set_err(c, SIDM_EINVAL, "null argument");
    c->step_bins = nullptr;
    return scatter_impl(c, seed, step, xs, dt, mass, vel, stats, s);
}

extern "C" int sidm_scatter_step_binned(sidm_ctx* c, uint64_t seed, uint64_t step, const sidm_xs* xs, double dt_max,
                                        int32_t n_bins, int32_t substep, const int32_t* bins, const double* mass,
                                        void* vel, sidm_step_stats* stats, cudaStream_t s)
{
    if (!c) return SIDM_EINVAL;
    if (!c->sized) return set_err(c, SIDM_EINVAL, "sidm_kernel_sizes must come first");
    if (!xs || !mass || ((!vel || !bins) && c->lay.N > 0)) return set_err(c, SIDM_EINVAL, "null argument");
    if (n_bins < 1 || n_bins > 16) return set_err(c, SIDM_EINVAL, "n_bins must be in 1..16");
    if (substep < 0 || substep >= (1 << (n_bins - 1))) return set_err(c, SIDM_EINVAL, "substep out of range");
    if (!(dt_max > 0.0)) return set_err(c, SIDM_EINVAL, "dt_max must be positive");
    c->step_bins = bins;
    c->step_nbins = n_bins;
    c->step_sub = substep;
    c->step_dtmax = dt_max;
    const int rc = scatter_impl(c, seed, step, xs, nullptr, mass, vel, stats, s);
    c->step_bins = nullptr;
    return rc;
}

constexpr double kPiD = 3.14159265358979323846;

// Analytic host galaxy (Sect. 4.1): NFW halo, Hernquist bulge and up to four
// Miyamoto-Nagai disks, in FP64.  d = x - centre.  The acceleration is the
// hand-differentiated -grad Phi of each part:
//   spherical parts: -G [M_NFW(<r) / r^3 + M_H / (r (r + a_H)^2)] d,
//                    M_NFW(<r) = 4 pi rho_s r_s^3 (ln(1 + u) - u / (1 + u)), u = r / r_s;
//   disk:            -G M_d D^(-3/2) (dx, dy, dz (a_d + zeta) / zeta),
//                    zeta = sqrt(dz^2 + b_d^2), D = R^2 + (a_d + zeta)^2.
__device__ __forceinline__ void host_accel(const sidm_host& H, double dx, double dy, double dz, double& ax,
                                           double& ay, double& az)
{
    const double R2 = dx * dx + dy * dy;
    const double r2 = R2 + dz * dz;
    ax = ay = az = 0.0;
    if (r2 > 0.0) {
        const double r = sqrt(r2);
        double f = 0.0;
        if (H.rho_s != 0.0) {
            const double u = r / H.r_s;
            const double m = 4.0 * kPiD * H.rho_s * H.r_s * H.r_s * H.r_s * (log1p(u) - u / (1.0 + u));
            f += m / (r2 * r);
        }
        if (H.M_H != 0.0) {
            const double ra = r + H.a_H;
            f += H.M_H / (r * ra * ra);
        }
        ax = -H.G * f * dx; ay = -H.G * f * dy; az = -H.G * f * dz;
    }
    for (int k = 0; k < H.n_disks; ++k) {
        const double zeta = sqrt(dz * dz + H.b_d[k] * H.b_d[k]);
        const double sz = H.a_d[k] + zeta;
        const double rd = rsqrt(R2 + sz * sz);
        const double f = -H.G * H.M_d[k] * rd * rd * rd;
        ax += f * dx;
        ay += f * dy;
        az += f * dz * (sz / zeta);
    }
}

__device__ __forceinline__ double host_phi(const sidm_host& H, double dx, double dy, double dz)
{
    const double R2 = dx * dx + dy * dy;
    const double r = sqrt(R2 + dz * dz);
    double phi = 0.0;
    if (H.rho_s != 0.0) {
        const double k = 4.0 * kPiD * H.G * H.rho_s * H.r_s * H.r_s * H.r_s;
        phi -= (r > 0.0) ? k * log1p(r / H.r_s) / r : k / H.r_s;
    }
    if (H.M_H != 0.0) phi -= H.G * H.M_H / (r + H.a_H);
    for (int k = 0; k < H.n_disks; ++k) {
        const double sz = H.a_d[k] + sqrt(dz * dz + H.b_d[k] * H.b_d[k]);
        phi -= H.G * H.M_d[k] * rsqrt(R2 + sz * sz);
    }
    return phi;
}

// Half kick by the analytic host for the particles whose individual step
// opens (phase 0) or closes (phase 1) at this sub-step; FP64 acceleration.
template <class R>
__global__ void k_host_kick(int64_t N, const double* __restrict__ pos, R* __restrict__ vel,
                            const int32_t* __restrict__ bins, int n_bins, int substep, int phase, double dt_max,
                            const sidm_host H)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = bins ? bins[i] : 0;
        const int period = 1 << (n_bins - 1 - b);
        const bool due = phase == 0 ? (substep % period == 0) : ((substep + 1) % period == 0);
        if (!due) continue;
        double ax, ay, az;
        host_accel(H, pos[i] - H.center[0], pos[N + i] - H.center[1], pos[2 * N + i] - H.center[2], ax, ay, az);
        const double hdt = 0.5 * ldexp(dt_max, -b);
        vel[i] = (R)((double)vel[i] + ax * hdt);
        vel[N + i] = (R)((double)vel[N + i] + ay * hdt);
        vel[2 * N + i] = (R)((double)vel[2 * N + i] + az * hdt);
    }
}

__global__ void k_host_potential(int64_t N, const double* __restrict__ pos, double* __restrict__ phi,
                                 const sidm_host H)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        phi[i] = host_phi(H, pos[i] - H.center[0], pos[N + i] - H.center[1], pos[2 * N + i] - H.center[2]);
}

static bool host_ok(const sidm_host* h)
{
    if (!(h->G >= 0.0) || !(h->rho_s >= 0.0) || !(h->r_s > 0.0) || !(h->M_H >= 0.0) || !(h->a_H > 0.0)) return false;
    if (h->n_disks < 0 || h->n_disks > SIDM_HOST_MAX_DISKS) return false;
    for (int k = 0; k < h->n_disks; ++k)
        if (!(h->M_d[k] >= 0.0) || !(h->a_d[k] >= 0.0) || !(h->b_d[k] > 0.0)) return false;
    for (int k = 0; k < 3; ++k)
        if (!isfinite(h->center[k])) return false;
    return true;
}

extern "C" int sidm_host_kick(sidm_ctx* c, const sidm_host* host, double dt_max, int32_t n_bins, int32_t substep,
                              int32_t phase, const int32_t* bins, const double* pos, void* vel, cudaStream_t s)
{
    if (!c) return SIDM_EINVAL;
    if (!c->has_layout) return set_err(c, SIDM_EINVAL, "sidm_build_cells must come first");
    if (!host || ((!pos || !vel) && c->lay.N > 0)) return set_err(c, SIDM_EINVAL, "null argument");
    if (n_bins < 1 || n_bins > 16) return set_err(c, SIDM_EINVAL, "n_bins must be in 1..16");
    if (substep < 0 || substep >= (1 << (n_bins - 1))) return set_err(c, SIDM_EINVAL, "substep out of range");
    if (phase != 0 && phase != 1) return set_err(c, SIDM_EINVAL, "phase must be 0 (opening) or 1 (closing)");
    if (!(dt_max > 0.0) || !host_ok(host)) return set_err(c, SIDM_EINVAL, "bad host or dt_max");
    SIDM_CUDA(c, ensure_device(c));
    const int64_t N = c->lay.N;
    if (N == 0) return SIDM_OK;
    if (c->cfg.precision == SIDM_FP64)
        SIDM_LAUNCH(c, k_host_kick<double><<<grid_for(c, N, 256), 256, 0, s>>>(N, pos, (double*)vel, bins, n_bins, substep,
                                                                              phase, dt_max, *host));
    else
        SIDM_LAUNCH(c, k_host_kick<float><<<grid_for(c, N, 256), 256, 0, s>>>(N, pos, (float*)vel, bins, n_bins, substep,
                                                                             phase, dt_max, *host));
    return SIDM_OK;
}

extern "C" int sidm_host_potential(sidm_ctx* c, const sidm_host* host, const double* pos, double* phi, cudaStream_t s)
{
    if (!c) return SIDM_EINVAL;
    if (!c->has_layout) return set_err(c, SIDM_EINVAL, "sidm_build_cells must come first");
    if (!host || ((!pos || !phi) && c->lay.N > 0)) return set_err(c, SIDM_EINVAL, "null argument");
    if (!host_ok(host)) return set_err(c, SIDM_EINVAL, "bad host");
    SIDM_CUDA(c, ensure_device(c));
    const int64_t N = c->lay.N;
    if (N == 0) return SIDM_OK;
    SIDM_LAUNCH(c, k_host_potential<<<grid_for(c, N, 256), 256, 0, s>>>(N, pos, phi, *host));
    return SIDM_OK;
}

extern "C" int sidm_energy_momentum(sidm_ctx* c, const double* mass, const void* vel, double* out, double* comp,
                                    cudaStream_t s)
{
    if (!c) return SIDM_EINVAL;
    if (!c->has_layout) return set_err(c, SIDM_EINVAL, "sidm_build_cells must come first");
    if (!mass || !out || (!vel && c->lay.N > 0)) return set_err(c, SIDM_EINVAL, "null argument");
    SIDM_CUDA(c, ensure_device(c));
    const LayoutHost& L = c->lay;
    if (L.nchunk > 0) {
        if (c->cfg.precision == SIDM_FP64)
            SIDM_LAUNCH(c, k_energy_partial<double><<<L.nchunk, sidm_sum::chunk_threads<double>(), 0, s>>>(
                (const double*)vel, L.N, c->d_chunk_halo, c->d_chunk_begin, c->d_halo_off, c->d_epart));
        else
            SIDM_LAUNCH(c, k_energy_partial<float><<<L.nchunk, sidm_sum::chunk_threads<float>(), 0, s>>>(
                (const float*)vel, L.N, c->d_chunk_halo, c->d_chunk_begin, c->d_halo_off, c->d_epart));
    }
    if (L.ngroup > 0)
        SIDM_LAUNCH(c, k_energy_group<<<(L.ngroup + 3) / 4, 128, 0, s>>>(L.H, L.ngroup, c->d_group_off, c->d_chunk_off,
                                                                         c->d_epart, c->d_gpart));
    SIDM_LAUNCH(c, k_energy_final<<<(L.H + 3) / 4, 128, 0, s>>>(L.H, c->d_group_off, mass, c->d_gpart, out, comp));
    return SIDM_OK;
}

extern "C" int sidm_status(sidm_ctx* c, cudaStream_t s, uint32_t* status)
{
    if (!c) return SIDM_EINVAL;
    SIDM_CUDA(c, ensure_device(c));
    SIDM_CUDA(c, cudaStreamSynchronize(s));
    unsigned int v = 0;
    SIDM_CUDA(c, cudaMemcpy(&v, &c->d_cnt->status, sizeof(v), cudaMemcpyDeviceToHost));
    SIDM_CUDA(c, cudaMemset(&c->d_cnt->status, 0, sizeof(v)));
    if (status) *status = v;
    if (v) {
        std::string m = "device status";
        if (v & SIDM_DEV_EVENT_OVERFLOW) m += " event-overflow";
        if (v & SIDM_DEV_ROUNDS) m += " round-limit";
        if (v & SIDM_DEV_STACK) m += " traversal-stack";
        if (v & SIDM_DEV_BAD_INPUT) m += " bad-input";
        if (v & SIDM_DEV_WAIT_TIMEOUT) m += " wait-timeout";
        return set_err(c, SIDM_EDEVICE, m);
    }
    return SIDM_OK;
}

extern "C" int sidm_get_perm(sidm_ctx* c, uint32_t* perm, cudaStream_t s)
{
    if (!c) return SIDM_EINVAL;
    if (!c->built) return set_err(c, SIDM_EINVAL, "sidm_build_cells must come first");
    if (!perm) return set_err(c, SIDM_EINVAL, "null argument");
    SIDM_CUDA(c, ensure_device(c));
    if (c->lay.N) SIDM_CUDA(c, cudaMemcpyAsync(perm, c->d_perm, sizeof(uint32_t) * c->lay.N, cudaMemcpyDeviceToDevice, s));
    return SIDM_OK;
}

extern "C" int sidm_get_events(sidm_ctx* c, int64_t cap, sidm_event* ev, int64_t* n_host, cudaStream_t s)
{
    if (!c) return SIDM_EINVAL;
    if (!c->stepped) return set_err(c, SIDM_EINVAL, "sidm_scatter_step must come first");
    if (!n_host || (cap > 0 && !ev)) return set_err(c, SIDM_EINVAL, "null argument");
    SIDM_CUDA(c, ensure_device(c));
    SIDM_CUDA(c, cudaStreamSynchronize(s));
    unsigned long long n = 0;
    SIDM_CUDA(c, cudaMemcpy(&n, &c->d_cnt->ev_count, sizeof(n), cudaMemcpyDeviceToHost));
    *n_host = (int64_t)n;
    const int64_t m = std::min<int64_t>({(int64_t)n, cap, c->cfg.event_cap});
    if (m > 0) SIDM_CUDA(c, cudaMemcpy(ev, c->d_ev, sizeof(sidm_event) * m, cudaMemcpyDeviceToDevice));
    return SIDM_OK;
}

extern "C" int sidm_lambda_eval(sidm_ctx* c, int64_t n, const double* d, const double* hi, const double* hj,
                                double* out, cudaStream_t s)
{
    if (!c) return SIDM_EINVAL;
    if (n < 0 || (n > 0 && (!d || !hi || !hj || !out))) return set_err(c, SIDM_EINVAL, "bad argument");
    if (n == 0) return SIDM_OK;
    SIDM_CUDA(c, ensure_device(c));
    if (c->cfg.precision == SIDM_FP64)
        SIDM_LAUNCH(c, k_lambda_eval<double><<<grid_for(c, n, 256), 256, 0, s>>>(n, d, hi, hj, out, (const double*)c->d_lam));
    else
        SIDM_LAUNCH(c, k_lambda_eval<float><<<grid_for(c, n, 256), 256, 0, s>>>(n, d, hi, hj, out, (const float*)c->d_lam));
    return SIDM_OK;
}

extern "C" int sidm_drift(sidm_ctx* c, const double* dt, double* pos, const void* vel, cudaStream_t s)
{
    if (!c) return SIDM_EINVAL;
    if (!c->has_layout) return set_err(c, SIDM_EINVAL, "sidm_build_cells must come first");
    if (!dt || (c->lay.N > 0 && (!pos || !vel))) return set_err(c, SIDM_EINVAL, "null argument");
    if (c->lay.N == 0) return SIDM_OK;
    SIDM_CUDA(c, ensure_device(c));
    if (c->cfg.precision == SIDM_FP64)
        SIDM_LAUNCH(c, k_drift<double><<<grid_for(c, c->lay.N, 256), 256, 0, s>>>(c->lay.N, c->lay.H, c->d_halo_off, dt, pos,
                                                                                (const double*)vel));
    else
        SIDM_LAUNCH(c, k_drift<float><<<grid_for(c, c->lay.N, 256), 256, 0, s>>>(c->lay.N, c->lay.H, c->d_halo_off, dt, pos,
                                                                               (const float*)vel));
    return SIDM_OK;
}

extern "C" int sidm_reflect_boundary(sidm_ctx* c, const double* bound, const double* pos, void* vel, cudaStream_t s)
{
    if (!c) return SIDM_EINVAL;
    if (!c->has_layout) return set_err(c, SIDM_EINVAL, "sidm_build_cells must come first");
    if (!bound || (c->lay.N > 0 && (!pos || !vel))) return set_err(c, SIDM_EINVAL, "null argument");
    if (c->lay.N == 0) return SIDM_OK;
    SIDM_CUDA(c, ensure_device(c));
    if (c->cfg.precision == SIDM_FP64)
        SIDM_LAUNCH(c, k_reflect<double><<<grid_for(c, c->lay.N, 256), 256, 0, s>>>(c->lay.N, c->lay.H, c->d_halo_off,
                                                                                  bound, pos, (double*)vel));
    else
        SIDM_LAUNCH(c, k_reflect<float><<<grid_for(c, c->lay.N, 256), 256, 0, s>>>(c->lay.N, c->lay.H, c->d_halo_off,
                                                                                 bound, pos, (float*)vel));
    return SIDM_OK;
}

extern "C" int sidm_get_sum_p(sidm_ctx* c, float* out, cudaStream_t s)
{
    if (!c) return SIDM_EINVAL;
    if (!(c->cfg.flags & SIDM_FLAG_SUM_P)) return set_err(c, SIDM_EINVAL, "context built without SIDM_FLAG_SUM_P");
    if (!out) return set_err(c, SIDM_EINVAL, "null argument");
    SIDM_CUDA(c, ensure_device(c));
    if (c->lay.N) SIDM_CUDA(c, cudaMemcpyAsync(out, c->d_sump, sizeof(float) * c->lay.N, cudaMemcpyDeviceToDevice, s));
    return SIDM_OK;
}

extern "C" int sidm_kernel_times(sidm_ctx* c, double* ms, int64_t* count, int32_t reset)
{
    if (!c) return SIDM_EINVAL;
    if (!(c->cfg.flags & SIDM_FLAG_TIMING)) return set_err(c, SIDM_EINVAL, "context built without SIDM_FLAG_TIMING");
    if (!ms) return set_err(c, SIDM_EINVAL, "null argument");
    SIDM_CUDA(c, ensure_device(c));
    SIDM_CUDA(c, cudaDeviceSynchronize());
    for (int k = 0; k < 4; ++k) { ms[k] = 0.0; if (count) count[k] = 0; }
    for (int i = 0; i < c->t_used; ++i) {
        float t = 0.f;
        SIDM_CUDA(c, cudaEventElapsedTime(&t, c->t_ev[2 * i], c->t_ev[2 * i + 1]));
        ms[c->t_slot[i]] += (double)t;
        if (count) count[c->t_slot[i]] += 1;
    }
    if (reset) c->t_used = 0;
    return SIDM_OK;
}

extern "C" int sidm_warm_start(sidm_ctx* c, int32_t enable)
{
    if (!c) return SIDM_EINVAL;
    c->warm_enabled = enable != 0;
    if (!c->warm_enabled) c->hprev_valid = false;
    return SIDM_OK;
}

extern "C" int sidm_diagnostics(sidm_ctx* c, uint64_t* out, int32_t reset)
{
    if (!c) return SIDM_EINVAL;
    if (!out) return set_err(c, SIDM_EINVAL, "null argument");
    SIDM_CUDA(c, ensure_device(c));
    SIDM_CUDA(c, cudaDeviceSynchronize());
    SIDM_CUDA(c, cudaMemcpy(out, c->d_cnt->diag, sizeof(unsigned long long) * 8, cudaMemcpyDeviceToHost));
    if (reset) SIDM_CUDA(c, cudaMemset(c->d_cnt->diag, 0, sizeof(unsigned long long) * 8));
    return SIDM_OK;
}
