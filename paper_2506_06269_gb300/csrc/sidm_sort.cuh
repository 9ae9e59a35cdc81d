// sidm_sort.cuh -- stable LSD radix sort of (u64 key, u32 value) pairs with
// 8-bit digits, one launch per digit (a chained scan with decoupled
// look-back), used by the cell build (Morton keys) and by the per-particle
// interaction lists of the list resolve.
//
//   k_sort_count   one read of the keys: the digit counts of every pass at once
//                  ([passes][256], shared-memory atomics); the cell build takes
//                  them in the kernel that makes its keys instead.
//   k_sort_pass    one digit: persistent CTAs (two per SM) take tiles of
//                  kTile = 4096 keys in ticket order; the next tile's keys and
//                  values are copied into a staging buffer (two bulk
//                  asynchronous copies, TMA) while the current one is sorted.
//                  A tile is ranked per warp (warp w owns the tile's 512
//                  consecutive keys w*512 ..; eight ballots group equal digits
//                  of one round of 32), its digit counts are published at once,
//                  it is reordered by digit in shared memory, a look-back over
//                  the earlier tiles' published counts gives its exclusive
//                  prefix (8 words per round trip), and it is written out in
//                  runs of equal digits (coalesced).  Per key a pass moves 12
//                  bytes in and 12 out, the bytes of the pass.
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
constexpr int kItems = 16;                        // keys per thread
constexpr int kTile = kThreads * kItems;          // 4096 keys per tile
constexpr int kWarpKeys = 32 * kItems;            // 512 consecutive keys per warp
constexpr int kPassCtas = 2;                      // resident CTAs per SM the pass is built for
constexpr int kMaxPasses = 8;
constexpr unsigned long long kFlagA = 1ull << 62;  // tile count published
constexpr unsigned long long kFlagP = 2ull << 62;  // inclusive prefix published
constexpr unsigned long long kValMask = (1ull << 62) - 1ull;
constexpr unsigned long long kLookNs = 20000000ull;  // 20 ms per wait
constexpr unsigned kLookPolls = 1u << 22;

struct Smem {
    unsigned long long skey[kTile];     // staging of the next tile (bulk copies)
    uint32_t sval[kTile];
    unsigned long long key[kTile];      // the current tile in digit order
    uint32_t val[kTile];
    uint32_t wcnt[kWarps][256];     // per-warp digit counts, then their exclusive offsets
    long long off[256];             // global slot of the tile's first key of each digit, minus its tile slot
    uint32_t tstart[256];           // tile slot of the first key of each digit
    uint32_t wsum[kWarps];
    unsigned long long bar;             // mbarrier of the staging copies
    int next;                           // the CTA's next ticket
    int late;                           // a staging wait gave up: plain loads from then on
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

// One tile of one digit pass, its keys and values in registers (k, v; slot
// r of lane l of warp w is tile key w*kWarpKeys + r*32 + l).  Ranks per warp,
// publishes the tile's counts, reorders the tile in shared memory, looks back
// for the exclusive prefix and writes the tile out.  Called by all threads;
// S.wcnt must be zero on entry.
__device__ __forceinline__ void sort_tile(Smem& S, const unsigned long long (&k)[kItems], const uint32_t (&v)[kItems],
                                          int tile, int64_t n, int shift, const uint32_t* __restrict__ cnt,
                                          unsigned long long* __restrict__ status, unsigned long long* __restrict__ kout,
                                          uint32_t* __restrict__ vout, unsigned int* err, unsigned int err_bit)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t t0 = (int64_t)tile * kTile;
    const int64_t wbase = t0 + warp * kWarpKeys;
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

// One digit pass: kin/vin -> kout/vout by digit (key >> shift) & 255.
// Persistent CTAs (grid <= tiles) take tiles in ticket order; while a CTA
// sorts one tile, the next one's keys and values are already on their way
// into a staging buffer by two bulk asynchronous copies (TMA, one thread,
// completion counted on an mbarrier).  The wait is bounded: on expiry the
// status bit is raised, no copy is issued any more, tiles are read with plain
// loads, and the CTA waits (again bounded) for the late copy before it exits.
// A tile whose copy would not be whole (the last one, when n is not a
// multiple of kTile, or every tile when kin or vin is not 16-byte aligned) is
// read with plain loads.  cnt = this pass's 256 digit
// totals; status [tiles][256] and *ticket zero on entry; dynamic shared
// memory kSmemBytes.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t ph)
{
    const unsigned long long t0 = now_ns();
    for (unsigned it = 0; it < kLookPolls; ++it) {
        uint32_t r;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(r) : "r"(bar), "r"(ph) : "memory");
        if (r) return true;
        if (now_ns() - t0 > kLookNs) return false;
    }
    return false;
}

__global__ void __launch_bounds__(kThreads, kPassCtas) k_sort_pass(const unsigned long long* __restrict__ kin,
                                                           const uint32_t* __restrict__ vin, int64_t n, int shift,
                                                           int tiles, bool bulk, const uint32_t* __restrict__ cnt,
                                                           unsigned long long* __restrict__ status,
                                                           unsigned int* __restrict__ ticket,
                                                           unsigned long long* __restrict__ kout,
                                                           uint32_t* __restrict__ vout, unsigned int* __restrict__ err,
                                                           unsigned int err_bit)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&S.bar);
    // thread 0: the copies of tile tl into the staging buffer
    auto issue = [&](int tl) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"((uint32_t)(kTile * 12)) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"((uint32_t)__cvta_generic_to_shared(S.skey)), "l"(kin + (int64_t)tl * kTile),
                     "r"((uint32_t)(kTile * 8)), "r"(bar) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"((uint32_t)__cvta_generic_to_shared(S.sval)), "l"(vin + (int64_t)tl * kTile),
                     "r"((uint32_t)(kTile * 4)), "r"(bar) : "memory");
    };
    // bulk: kin and vin 16-byte aligned (a copy must start on a 16-byte boundary)
    auto whole = [&](int tl) { return bulk && (int64_t)(tl + 1) * kTile <= n; };
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.next = (int)atomicAdd(ticket, 1u);
        S.late = 0;
        if (S.next < tiles && whole(S.next)) issue(S.next);
    }
    __syncthreads();
    int tile = S.next;
    uint32_t phase = 0u;
    bool staged = tile < tiles && whole(tile);
    bool pending = false;                      // a copy gave up on may still land
    while (tile < tiles) {
        unsigned long long k[kItems];
        uint32_t v[kItems];
        bool from_stage = false;
        if (staged) {
            const bool ok = __syncthreads_and(bar_wait(bar, phase));
            if (ok) {
                phase ^= 1u;
                from_stage = true;
            } else {
                pending = true;
                if (t == 0) { S.late = 1; atomicOr(err, err_bit); }
            }
        }
        const int64_t wbase = (int64_t)tile * kTile + warp * kWarpKeys;
#pragma unroll
        for (int r = 0; r < kItems; ++r) {
            const int li = warp * kWarpKeys + r * 32 + lane;
            const int64_t s = wbase + r * 32 + lane;
            k[r] = from_stage ? S.skey[li] : (s < n ? kin[s] : 0ull);
            v[r] = from_stage ? S.sval[li] : (s < n ? vin[s] : 0u);
        }
#pragma unroll
        for (int w = 0; w < kWarps; ++w) S.wcnt[w][t] = 0u;
        __syncthreads();                       // staging buffer read, S.next free
        if (t == 0) {
            S.next = (int)atomicAdd(ticket, 1u);
            if (!S.late && S.next < tiles && whole(S.next)) issue(S.next);
        }
        __syncthreads();
        const int next = S.next;
        const bool next_staged = !S.late && next < tiles && whole(next);
        sort_tile(S, k, v, tile, n, shift, cnt, status, kout, vout, err, err_bit);
        __syncthreads();                       // S.key / S.off / S.wcnt reused by the next tile
        tile = next;
        staged = next_staged;
    }
    // a copy whose wait gave up may still be writing this CTA's shared memory
    if (pending) {
        const bool ok = __syncthreads_and(bar_wait(bar, phase));
        if (!ok && t == 0) atomicOr(err, err_bit);
    }
}

}  // namespace sidm_sort
