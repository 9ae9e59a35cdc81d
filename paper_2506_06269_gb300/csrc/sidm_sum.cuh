// sidm_sum.cuh -- per-halo kinetic energy and momentum (step a5), shared by
// sidm_energy_momentum and sidm_energy_momentum_static so that the two give
// identical bits.
//
// Both reduce a halo in chunks of at most 16384 particles, one CTA per chunk
// (512 threads for FP32 velocities, 256 for FP64), to four unscaled sums
// S = (sum |v|^2, sum vx, sum vy, sum vz), each kept as a double-double
// (hi, lo).  The chunk sums are merged in a fixed order in two levels, so
// that the slow FP64 pipe of a single SM never takes a whole large halo: one
// warp per group of up to 32 consecutive chunks of a halo (lane i takes chunk
// i, then a fixed shuffle tree), then one warp per halo over its groups (lane
// l takes groups l, l+32, ... in turn, then the same tree), scaled by
// (m/2, m, m, m).
//
// FP32 velocities (the mixed form) are summed EXACTLY on the integer pipes.
// GB300 issues FP64 arithmetic at a small fraction of its FP32/INT32 rate, so
// a compensated FP64 sum costs more here than the whole integer route.  With
// E the largest binary exponent in the chunk, each x = m 2^(e-23) (m < 2^24)
// is an integer in units of 2^(E-111) and each x^2 = m^2 2^(2e-46) one in
// units of 2^(2E-110); a signed (linear terms) or unsigned (squares) 128-bit
// accumulator holds 2^14 such terms without overflow (|x| < 2^(E+1) is below
// 2^112 units, and so is x^2).  Only terms under 2^(E-88) and squares under
// 2^(2E-64) have bits below one unit; dropping them costs less than 2^-94 of
// the chunk's largest term in all.  Integer addition is associative, so the chunk sums do
// not depend on the order of the tree.  Each chunk's integer then becomes the
// double-double (RN(S), RN(S - RN(S))).
//
// Nearly every component lies within 2^16 of the chunk's largest (e >= E-16)
// or is zero; a thread sums those in narrower exact windows first: the
// linear terms as 64-bit integers in units of 2^(E-39) (m 2^(e-E+16) < 2^40,
// at most 32 per thread), the squares as 128-bit integers in units of
// 2^(2E-78) (below 2^80).  Shifted by 72 and 32 bits these are the same
// integers in the chunk's windows, so the sums are bit-identical; the others
// take the general route.
//
// FP64 velocities (the FP64 form) keep a compensated (two-sum) FP64 sum in a
// fixed order: thread t takes elements t, t+256, ..., then a fixed binary tree
// over the 256 threads.
#pragma once

#include <cstdint>

namespace sidm_sum {

constexpr int kThreadsF32 = 512;   // CTA of the exact FP32 chunk sums (two per SM at 54 registers)
constexpr int kThreadsF64 = 256;   // CTA of the compensated FP64 chunk sums
constexpr int kMaxChunk = 16384;   // the integer windows above hold 2^14 terms

template <class R> constexpr int chunk_threads() { return sizeof(R) == 4 ? kThreadsF32 : kThreadsF64; }

struct DD { double s, c; };

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e)
{
    s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

__device__ __forceinline__ void dd_add(DD& x, double v)
{
    double s, e;
    two_sum(x.s, v, s, e);
    x.s = s;
    x.c = __dadd_rn(x.c, e);
}

__device__ __forceinline__ void dd_merge(DD& x, const DD& y)
{
    double s, e;
    two_sum(x.s, y.s, s, e);
    x.s = s;
    x.c = __dadd_rn(__dadd_rn(x.c, y.c), e);
}

typedef unsigned __int128 u128;


// 64-bit shifts whose amount is taken unsigned and clamped at 64 (PTX shl/shr
// semantics): an amount of 64 or more, or a negative int, gives 0
__device__ __forceinline__ unsigned long long shl64(unsigned long long x, int n)
{
    unsigned long long r;
    asm("shl.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(n));
    return r;
}
__device__ __forceinline__ unsigned long long shr64(unsigned long long x, int n)
{
    unsigned long long r;
    asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(n));
    return r;
}

// x placed in the chunk's fixed-point windows: lin += x / 2^(E-111),
// sq += x^2 / 2^(2E-110), both truncated toward zero below one unit.
// The term t = M 2^o (o <= 88 for x, o2 <= 64 for x^2) is built as two 64-bit
// words with clamped shifts: lo = M << o | M >> -o (one of the two is 0), and
// hi = floor(t / 2^64) = (M << 40) >> (104 - o) for M < 2^24 (the square:
// (M2 << 16) >> (80 - o2) for M2 < 2^48); the shift amounts are >= 16.
__device__ __forceinline__ void exact_add(float x, int E, u128& lin, u128& sq)
{
    const uint32_t b = __float_as_uint(x);
    const uint32_t ex = (b >> 23) & 255u;
    const uint32_t m = (b & 0x7FFFFFu) | (ex ? 0x800000u : 0u);
    const int d = (int)(ex ? ex : 1u) - 127 - E;             // e - E <= 0
    const int o1 = 88 + d;
    const unsigned long long M = m;
    const u128 t = ((u128)shr64(M << 40, 104 - o1) << 64) | (shl64(M, o1) | shr64(M, -o1));
    lin += (b >> 31) ? (u128)0 - t : t;                      // two's complement
    const unsigned long long M2 = (unsigned long long)m * m;
    const int o2 = 64 + 2 * d;
    sq += ((u128)shr64(M2 << 16, 80 - o2) << 64) | (shl64(M2, o2) | shr64(M2, -o2));
}

// Thread-level narrow windows of the components with e >= E - 16 (or zero):
// lin += x / 2^(E-39), sq += x^2 / 2^(2E-78), exact; the rest go to the chunk
// windows through exact_add.
struct NarrowSums {
    long long lx = 0, ly = 0, lz = 0;
    u128 sq = 0;
};
__device__ __forceinline__ void narrow_add(float x, int E, long long& lin, NarrowSums& ns, u128& wide_lin,
                                           u128& wide_sq)
{
    const uint32_t b = __float_as_uint(x);
    const uint32_t ex = (b >> 23) & 255u;
    const uint32_t m = (b & 0x7FFFFFu) | (ex ? 0x800000u : 0u);
    const int s1 = (int)ex - 127 - E + 16;                   // e - E + 16 for normal x
    if (ex != 0u && s1 >= 0) {
        const unsigned long long tu = (unsigned long long)m << s1;   // < 2^40
        const long long t = (long long)tu;
        lin += (b >> 31) ? -t : t;
        // x^2 / 2^(2E-78) = t^2 < 2^80: a 64 x 64 -> 128-bit product (multiply
        // pipe, not the shift/logic pipe the rest of this sum keeps busy)
        ns.sq += ((u128)__umul64hi(tu, tu) << 64) | (tu * tu);
    } else if (m != 0u) {
        exact_add(x, E, wide_lin, wide_sq);
    }
}

__device__ __forceinline__ u128 shfl_down_u128(u128 v, int o)
{
    const unsigned long long lo = __shfl_down_sync(0xffffffffu, (unsigned long long)v, o);
    const unsigned long long hi = __shfl_down_sync(0xffffffffu, (unsigned long long)(v >> 64), o);
    return ((u128)hi << 64) | lo;
}

// correctly rounded conversion of a 128-bit unsigned integer
__device__ __forceinline__ double u128_rn(u128 a)
{
    const unsigned long long hi = (unsigned long long)(a >> 64);
    if (hi == 0ull) return __ull2double_rn((unsigned long long)a);
    const int k = 64 - __clzll((long long)hi);               // bit length of a is 64 + k
    const unsigned long long top = (unsigned long long)(a >> k);
    const bool sticky = (a & (((u128)1 << k) - 1)) != 0;     // shifted-out bits join the sticky bit
    return ldexp(__ull2double_rn(top | (sticky ? 1ull : 0ull)), k);
}

// a non-negative integral double below 2^128 as an integer
__device__ __forceinline__ u128 dbl_to_u128(double h)
{
    if (h < 0x1p64) return (u128)__double2ull_rn(h);
    const unsigned long long bits = (unsigned long long)__double_as_longlong(h);
    const int ex = (int)((bits >> 52) & 2047ull) - 1075;     // h = mant 2^ex, ex >= 12
    const unsigned long long mant = (bits & ((1ull << 52) - 1ull)) | (1ull << 52);
    return (u128)mant << ex;
}

// the 128-bit integer v (two's complement if is_signed) times 2^L as (hi, lo)
__device__ __forceinline__ DD int_to_dd(u128 v, bool is_signed, int L)
{
    const bool neg = is_signed && (long long)(v >> 64) < 0;
    const u128 a = neg ? (u128)0 - v : v;
    const double h = u128_rn(a);
    const u128 H = dbl_to_u128(h);
    const double l = a >= H ? u128_rn(a - H) : -u128_rn(H - a);
    const double sgn = neg ? -1.0 : 1.0;
    return DD{ldexp(sgn * h, L), ldexp(sgn * l, L)};
}

// One chunk [b, e) of FP32 velocities [3][N]: exact sums, written as
// out8 = (S2 hi, S2 lo, Sx hi, Sx lo, Sy hi, Sy lo, Sz hi, Sz lo).
// Called by all kThreadsF32 threads of the CTA; e - b <= kMaxChunk.
__device__ __forceinline__ void chunk_sums(const float* __restrict__ vel, int64_t N, int64_t b, int64_t e,
                                           double* __restrict__ out8)
{
    constexpr int kThreads = kThreadsF32, kWarps = kThreadsF32 / 32;
    __shared__ uint32_t s_max[kWarps];
    __shared__ u128 s_part[kWarps][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the largest |bit pattern| has the largest exponent field (an infinity or
    // NaN gives 255)
    uint32_t mb = 0u;
#pragma unroll 8
    for (int64_t s = b + threadIdx.x; s < e; s += kThreads)
        mb = max(mb, max(__float_as_uint(vel[s]) & 0x7FFFFFFFu,
                         max(__float_as_uint(vel[N + s]) & 0x7FFFFFFFu, __float_as_uint(vel[2 * N + s]) & 0x7FFFFFFFu)));
    uint32_t mx = __reduce_max_sync(0xffffffffu, mb) >> 23;
    if (lane == 0) s_max[warp] = mx;
    __syncthreads();
    uint32_t M = 0u;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) M = max(M, s_max[w]);
    if (M == 255u) {                                         // an infinity or a NaN: no finite sum
        if (threadIdx.x < 8) out8[threadIdx.x] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const int E = (int)(M ? M : 1u) - 127;
    u128 sq = 0, lx = 0, ly = 0, lz = 0;
    NarrowSums ns;
#pragma unroll 4
    for (int64_t s = b + threadIdx.x; s < e; s += kThreads) {
        narrow_add(vel[s], E, ns.lx, ns, lx, sq);
        narrow_add(vel[N + s], E, ns.ly, ns, ly, sq);
        narrow_add(vel[2 * N + s], E, ns.lz, ns, lz, sq);
    }
    // narrow windows into the chunk's: x 2^72 (linear, sign-extended), x 2^32 (squares)
    lx += (u128)(__int128)ns.lx << 72;
    ly += (u128)(__int128)ns.ly << 72;
    lz += (u128)(__int128)ns.lz << 72;
    sq += ns.sq << 32;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sq += shfl_down_u128(sq, o);
        lx += shfl_down_u128(lx, o);
        ly += shfl_down_u128(ly, o);
        lz += shfl_down_u128(lz, o);
    }
    if (lane == 0) { s_part[warp][0] = sq; s_part[warp][1] = lx; s_part[warp][2] = ly; s_part[warp][3] = lz; }
    __syncthreads();
    if (threadIdx.x < 4) {
        const int a = threadIdx.x;
        u128 v = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) v += s_part[w][a];
        const DD r = a == 0 ? int_to_dd(v, false, 2 * E - 110) : int_to_dd(v, true, E - 111);
        out8[2 * a] = r.s;
        out8[2 * a + 1] = r.c;
    }
}

// One chunk [b, e) of FP64 velocities: compensated sums in a fixed order.
// Called by all kThreadsF64 threads of the CTA.
__device__ __forceinline__ void chunk_sums(const double* __restrict__ vel, int64_t N, int64_t b, int64_t e,
                                           double* __restrict__ out8)
{
    constexpr int kThreads = kThreadsF64;
    __shared__ DD sh[4][kThreads];
    DD acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int64_t s = b + threadIdx.x; s < e; s += kThreads) {
        const double x = vel[s], y = vel[N + s], z = vel[2 * N + s];
        double q = __dmul_rn(x, x);
        q = __dadd_rn(q, __dmul_rn(y, y));
        q = __dadd_rn(q, __dmul_rn(z, z));
        dd_add(acc[0], q);
        dd_add(acc[1], x);
        dd_add(acc[2], y);
        dd_add(acc[3], z);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) sh[a][threadIdx.x] = acc[a];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int a = 0; a < 4; ++a) dd_merge(sh[a][threadIdx.x], sh[a][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x < 4) {
        out8[2 * threadIdx.x] = sh[threadIdx.x][0].s;
        out8[2 * threadIdx.x + 1] = sh[threadIdx.x][0].c;
    }
}

__device__ __forceinline__ DD shfl_down_dd(const DD& x, int o)
{
    return DD{__shfl_down_sync(0xffffffffu, x.s, o), __shfl_down_sync(0xffffffffu, x.c, o)};
}

constexpr int kGroupChunks = 32;   // chunks per first-level group

// Chunks part[c0 .. c1) (c1 - c0 <= kGroupChunks) of one halo merged by one
// warp: lane i takes chunk c0 + i, then lane i takes lane i+16, i+8, ...;
// out8 = the group's four double-doubles.  Called by all 32 lanes of a warp.
__device__ __forceinline__ void group_sums(const double* __restrict__ part, int c0, int c1, double* __restrict__ out8)
{
    const int lane = threadIdx.x & 31;
    DD acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    if (c0 + lane < c1)
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a] = DD{part[(c0 + lane) * 8 + 2 * a], part[(c0 + lane) * 8 + 2 * a + 1]};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int a = 0; a < 4; ++a) dd_merge(acc[a], shfl_down_dd(acc[a], o));
    if (lane == 0)
#pragma unroll
        for (int a = 0; a < 4; ++a) { out8[2 * a] = acc[a].s; out8[2 * a + 1] = acc[a].c; }
}

// A halo's group sums part[c0 .. c1) merged by one warp in a fixed order
// (lane l: chunks c0+l, c0+l+32, ...; then lane i takes lane i+16, i+8, ...),
// then out = (m/2 S2, m Sx, m Sy, m Sz) and comp the rounding residual of
// each.  Called by all 32 lanes of a warp.
__device__ __forceinline__ void halo_result(const double* __restrict__ part, int c0, int c1, double m,
                                            double* __restrict__ out4, double* __restrict__ comp4)
{
    const int lane = threadIdx.x & 31;
    DD acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int c = c0 + lane; c < c1; c += 32)
#pragma unroll
        for (int a = 0; a < 4; ++a) dd_merge(acc[a], DD{part[c * 8 + 2 * a], part[c * 8 + 2 * a + 1]});
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int a = 0; a < 4; ++a) dd_merge(acc[a], shfl_down_dd(acc[a], o));
    if (lane == 0)                                         // only lane 0 holds the whole tree
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const double k = a == 0 ? __dmul_rn(0.5, m) : m;
            const double t = __dmul_rn(k, acc[a].c);
            const double v = __fma_rn(k, acc[a].s, t);
            out4[a] = v;
            if (comp4) comp4[a] = __dadd_rn(__fma_rn(k, acc[a].s, -v), t);
        }
}

}  // namespace sidm_sum
