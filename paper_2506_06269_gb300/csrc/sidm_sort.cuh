// sidm_sort.cuh -- stable LSD radix sort of (u64 key, u32 value) pairs with
// 8-bit digits, one launch per digit (a chained scan with decoupled
// look-back), used by the cell build (Morton keys) and by the per-particle
// interaction lists of the list resolve.
//
//   k_sort_count   one read of the keys: the digit counts of every pass at once
//                  ([passes][256], shared-memory atomics); the cell build takes
//                  them in the kernel that makes its keys instead.
//   k_sort_pass    one digit: a CTA takes the next tile of kTile = 2048 keys in
//                  ticket order, holds its keys and values in registers, ranks
//                  them per warp (warp w owns the tile's 256 consecutive keys
//                  w*256 ..; eight ballots group equal digits of one round of
//                  32), publishes its digit counts at once, reorders the tile by
//                  digit in shared memory, looks back over the earlier tiles'
//                  published counts for its exclusive prefix (8 words per round
//                  trip) and writes the tile out in runs of equal digits
//                  (coalesced).  Per key it moves 12 bytes in and 12 out, the
//                  bytes of the pass.
//
// Stability: inside a tile a key's rank among equal digits counts earlier
// warps, earlier rounds of its warp and earlier lanes of its round, i.e. the
// keys before it in index order; tiles are ranked in ticket order, and ticket
// t covers keys [t*kTile, (t+1)*kTile).
//
// Look-back: tile t writes (flag A | count) for each digit, then walks back
// over tiles t-1, t-2, ... adding counts until it meets an inclusive prefix
// (flag P), and writes (flag P | prefix + count).  A tile with a smaller
// ticket started earlier, is resident or done and publishes its counts before
// it waits on anything, so every wait ends; each wait is still bounded (poll
// count and %globaltimer), and on expiry raises a status bit and goes on.
#pragma once

#include <cstdint>

namespace sidm_sort {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;                         // keys per thread
constexpr int kTile = kThreads * kItems;          // 2048 keys per tile
constexpr int kWarpKeys = 32 * kItems;            // 256 consecutive keys per warp
constexpr int kPassCtas = kItems <= 8 ? 4 : 2;    // resident CTAs per SM the pass is built for
constexpr int kMaxPasses = 8;
constexpr unsigned long long kFlagA = 1ull << 62;  // tile count published
constexpr unsigned long long kFlagP = 2ull << 62;  // inclusive prefix published
constexpr unsigned long long kValMask = (1ull << 62) - 1ull;
constexpr unsigned long long kLookNs = 20000000ull;  // 20 ms per wait
constexpr unsigned kLookPolls = 1u << 22;

struct Smem {
    unsigned long long key[kTile];
    uint32_t val[kTile];
    uint32_t wcnt[kWarps][256];     // per-warp digit counts, then their exclusive offsets
    long long off[256];             // global slot of the tile's first key of each digit, minus its tile slot
    uint32_t tstart[256];           // tile slot of the first key of each digit
    uint32_t wsum[kWarps];
    int tile;
};
constexpr size_t kSmemBytes = sizeof(Smem);

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// exclusive scan of x over the 256 threads; *total receives the sum
__device__ __forceinline__ uint32_t exclusive256(uint32_t x, uint32_t* wsum, uint32_t* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t before = 0u, all = 0u;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t t = wsum[w];
        before += w < warp ? t : 0u;
        all += t;
    }
    __syncthreads();
    *total = all;
    return before + inc - x;
}

// Digit counts of passes 0 .. passes-1 over key[0, n); hist [passes][256]
// must be zero on entry.  Shared-memory atomics per key and pass, then one
// global atomic per CTA and nonzero count.
__device__ __forceinline__ void count_digits(uint32_t (*sh)[256], unsigned long long k, int passes)
{
    for (int p = 0; p < passes; ++p) atomicAdd(&sh[p][(uint32_t)(k >> (8 * p)) & 255u], 1u);
}

__global__ void __launch_bounds__(kThreads) k_sort_count(const unsigned long long* __restrict__ key, int64_t n,
                                                         int passes, uint32_t* __restrict__ hist)
{
    __shared__ uint32_t sh[kMaxPasses][256];
    for (int i = threadIdx.x; i < kMaxPasses * 256; i += kThreads) (&sh[0][0])[i] = 0u;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    int64_t s = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    for (; s + 3 * stride < n; s += 4 * stride) {
        unsigned long long k[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) k[r] = key[s + r * stride];
#pragma unroll
        for (int r = 0; r < 4; ++r) count_digits(sh, k[r], passes);
    }
    for (; s < n; s += stride) count_digits(sh, key[s], passes);
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += kThreads) {
        const uint32_t v = (&sh[0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
}

// Lanes of this warp (all 32 active) whose digit equals this lane's d (8 bits):
// one ballot per bit, lanes with valid = false match nobody.
__device__ __forceinline__ uint32_t match_digit(uint32_t d, bool valid)
{
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t v = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? v : ~v;
    }
    return peers;
}

// Walk back from tile j over the published words of digit column t until an
// inclusive prefix: kLookBatch words per round trip.  Returns the exclusive
// prefix; a wait past its bound raises err_bit and returns what it has.
constexpr int kLookBatch = 8;
__device__ __forceinline__ unsigned long long look_back(const unsigned long long* __restrict__ status, int j, int t,
                                                        unsigned int* err, unsigned int err_bit)
{
    unsigned long long excl = 0ull, since = 0ull;
    unsigned polls = 0u;
    while (j >= 0) {
        unsigned long long w[kLookBatch];
#pragma unroll
        for (int q = 0; q < kLookBatch; ++q)
            w[q] = j - q >= 0 ? ld_relaxed(status + (int64_t)(j - q) * 256 + t) : kFlagP;   // before tile 0: prefix 0
        int used = 0;
        bool done = false;
#pragma unroll
        for (int q = 0; q < kLookBatch; ++q) {
            if (done || used < q) break;                   // stopped at a word not yet published
            if (!(w[q] & (kFlagA | kFlagP))) break;
            excl += w[q] & kValMask;
            used = q + 1;
            if (w[q] & kFlagP) done = true;
        }
        if (done) return excl;
        j -= used;
        if (used == 0) {                                    // the next word is not published yet
            if (++polls == 64u) since = now_ns();
            if (polls > 64u && (polls & 255u) == 0u && (polls >= kLookPolls || now_ns() - since > kLookNs)) {
                atomicOr(err, err_bit);
                return excl;
            }
        }
    }
    return excl;
}

// One digit pass: kin/vin -> kout/vout by digit (key >> shift) & 255.
// cnt = this pass's 256 digit totals; status [tiles][256] and *ticket zero on
// entry; dynamic shared memory kSmemBytes.  The tile's counts are published
// as soon as they are known and the tile is reordered in shared memory (which
// frees the key registers) before the look-back.
__global__ void __launch_bounds__(kThreads, kPassCtas) k_sort_pass(const unsigned long long* __restrict__ kin,
                                                           const uint32_t* __restrict__ vin, int64_t n, int shift,
                                                           const uint32_t* __restrict__ cnt,
                                                           unsigned long long* __restrict__ status,
                                                           unsigned int* __restrict__ ticket,
                                                           unsigned long long* __restrict__ kout,
                                                           uint32_t* __restrict__ vout, unsigned int* __restrict__ err,
                                                           unsigned int err_bit)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) S.tile = (int)atomicAdd(ticket, 1u);
#pragma unroll
    for (int w = 0; w < kWarps; ++w) S.wcnt[w][t] = 0u;
    __syncthreads();
    const int tile = S.tile;
    const int64_t t0 = (int64_t)tile * kTile;
    const int64_t wbase = t0 + warp * kWarpKeys;
    unsigned long long k[kItems];
    uint32_t v[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int64_t s = wbase + r * 32 + lane;
        k[r] = s < n ? kin[s] : 0ull;
        v[r] = s < n ? vin[s] : 0u;
    }
    // rank among equal digits inside the warp's kWarpKeys keys
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t rk[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const bool ok = wbase + r * 32 + lane < n;
        const uint32_t d = (uint32_t)(k[r] >> shift) & 255u;
        const uint32_t peers = match_digit(d, ok);
        const uint32_t before = ok ? S.wcnt[warp][d] : 0u;
        rk[r] = before + (uint32_t)__popc(peers & lt);
        __syncwarp();
        if (ok && (peers & lt) == 0u) S.wcnt[warp][d] = before + (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // thread t owns digit t: offsets of the warps inside the tile's run of t,
    // the tile's count published at once
    uint32_t run = 0u;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = S.wcnt[w][t];
        S.wcnt[w][t] = run;
        run += c;
    }
    unsigned long long* mine = status + (int64_t)tile * 256 + t;
    st_relaxed(mine, (tile == 0 ? kFlagP : kFlagA) | run);
    uint32_t tile_total;
    const uint32_t tstart = exclusive256(run, S.wsum, &tile_total);
    S.tstart[t] = tstart;
    __syncthreads();
    // the tile in digit order in shared memory
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        if (wbase + r * 32 + lane < n) {
            const uint32_t d = (uint32_t)(k[r] >> shift) & 255u;
            const uint32_t pos = S.tstart[d] + S.wcnt[warp][d] + rk[r];
            S.key[pos] = k[r];
            S.val[pos] = v[r];
        }
    }
    uint32_t all;
    const uint32_t dbase = exclusive256(cnt[t], S.wsum, &all);
    // the keys of digit t in earlier tiles
    unsigned long long excl = 0ull;
    if (tile > 0) {
        excl = look_back(status, tile - 1, t, err, err_bit);
        st_relaxed(mine, kFlagP | (excl + run));
    }
    S.off[t] = (long long)dbase + (long long)excl - (long long)tstart;
    __syncthreads();
    const int64_t left = n - t0;
    const int tn = left < kTile ? (int)left : kTile;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int pos = i * kThreads + t;
        if (pos < tn) {
            const unsigned long long kk = S.key[pos];
            const int64_t dst = S.off[(uint32_t)(kk >> shift) & 255u] + pos;
            kout[dst] = kk;
            vout[dst] = S.val[pos];
        }
    }
}

}  // namespace sidm_sort
