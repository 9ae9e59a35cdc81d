// sidm_knn.cu -- (a1) kernel sizes: h_i = distance to the N_ngb-th nearest
// other particle of the halo (Sect. 2: each particle's kernel size adapts to
// its N_ngb nearest neighbours; Eq. hDl: h is the radius of the sphere holding
// N_ngb particles).
//
// One warp per leaf of 32 consecutive Morton-ordered particles, one query per
// lane.  Candidate leaves are staged through shared memory (plain coalesced
// 128-bit loads, or bulk asynchronous copies with an mbarrier), shifted into
// the query leaf's frame, and every lane keeps a 4-ary max-heap of its N_ngb
// smallest keys in shared memory (one 128-bit load per heap level).  The heap
// is first filled from the leaves next to the query leaf in Morton order
// (stored unsorted, then heapified once), whose k-th distance bounds the
// search radius; the bounding-volume tree is then walked with that
// (shrinking) radius, nearest children first, skipping those leaves.  Inside
// a tile a lane only appends keys below its current bound to a short pending
// list; the lists are merged into the heaps in batches, so the divergent heap
// sift runs with every lane busy instead of once per candidate.  The result
// is the exact k-th smallest of the canonical distance, so it does not depend
// on tile order, flush points or launch shape.
#include <type_traits>

#include "sidm_internal.cuh"
#include "sidm_tile.cuh"

namespace sidm {
namespace {

template <class R, bool NBR>
struct KeyOf {
    using T = typename std::conditional<(sizeof(R) == 8) || NBR, unsigned long long, uint32_t>::type;
};

struct KnnParams {
    int H, L;
    const int32_t* leaf_halo;
    const int32_t* leaf_off;
    const int64_t* halo_off;
    const int32_t* lvl_off;
    const int32_t* top;
    const int32_t* ngb;
    const HaloFrame* frame;
    const float4* cell;
    const float4* nlo;
    const float4* nhi;
    void* P4;
    const uint32_t* ID;
    void* h_out;
    uint32_t* nbr;
    int k_stride;
    int kcap;
    DevCounters* cnt;
    unsigned int* work;          // persistent work counter (zeroed before the launch)
    const int32_t* leaf_list;    // NULL: every leaf; else the leaves listed here ...
    const unsigned int* list_len;  // ... of which there are *list_len
    void* hprev;        // out: h per particle (next call's guess), NULL for neighbour lists
    int use_guess;      // P4.w holds each particle's previous kernel size
    float slack;        // guess bound = previous h * slack
    int flush_node;     // pending keys per lane that trigger a merge before a node's tests
};

template <class R, bool NBR>
__device__ __forceinline__ typename KeyOf<R, NBR>::T make_key(R d2, uint32_t id)
{
    if constexpr (sizeof(R) == 8) {
        return (unsigned long long)__double_as_longlong((double)d2);
    } else if constexpr (NBR) {
        return ((unsigned long long)__float_as_uint((float)d2) << 32) | id;
    } else {
        return __float_as_uint((float)d2);
    }
}

template <class R, bool NBR>
__device__ __forceinline__ R key_d2(typename KeyOf<R, NBR>::T k)
{
    if constexpr (sizeof(R) == 8) return (R)__longlong_as_double((long long)k);
    else if constexpr (NBR) return (R)__uint_as_float((uint32_t)(k >> 32));
    else return (R)__uint_as_float((uint32_t)k);
}

// Per-lane 4-ary max-heaps of keys (all keys are >= 0 as unsigned integers).
// Node t (0-based) sits at position t + 3, so the children 4t+1 .. 4t+4 of
// node t fill the aligned group t + 1.  Group g of lane l is stored at
// [g][l][0..3]: a lane reads all four children with one vector load and the
// 32 lanes of a warp hit distinct banks.  Positions past the last node read
// as 0, which never exceeds a key, so a missing child is never promoted.
template <class K>
struct Heap4 {
    K* g;        // [groups][32][4]
    int lane;
    __device__ K& at(int t) const { const int pos = t + 3; return g[((pos >> 2) * 32 + lane) * 4 + (pos & 3)]; }
    __device__ void children(int t, K c[4]) const
    {
        const K* src = g + ((t + 1) * 32 + lane) * 4;
        if constexpr (sizeof(K) == 4) {
            const uint4 v = *(const uint4*)src;
            c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
        } else {
            const ulonglong2 a = *(const ulonglong2*)src, b = *(const ulonglong2*)(src + 2);
            c[0] = a.x; c[1] = a.y; c[2] = b.x; c[3] = b.y;
        }
    }
    // zero the positions after node n-1 up to the end of its group
    __device__ void clear_tail(int n) const
    {
        for (int pos = n + 3; pos <= ((n + 2) | 3); ++pos) g[((pos >> 2) * 32 + lane) * 4 + (pos & 3)] = K(0);
    }
    // sift key down from node t of a heap of n nodes
    __device__ void sift(int t, int n, K key) const
    {
        while (4 * t + 1 < n) {
            K c[4];
            children(t, c);
            K m = c[0];
            int j = 0;
            if (c[1] > m) { m = c[1]; j = 1; }
            if (c[2] > m) { m = c[2]; j = 2; }
            if (c[3] > m) { m = c[3]; j = 3; }
            if (!(m > key)) break;
            at(t) = m;
            t = 4 * t + 1 + j;
        }
        at(t) = key;
    }
    // as sift, for a heap whose storage past node n-1 holds stale keys
    __device__ void sift_masked(int t, int n, K key) const
    {
        while (4 * t + 1 < n) {
            K c[4];
            children(t, c);
            if (4 * t + 2 >= n) c[1] = K(0);
            if (4 * t + 3 >= n) c[2] = K(0);
            if (4 * t + 4 >= n) c[3] = K(0);
            K m = c[0];
            int j = 0;
            if (c[1] > m) { m = c[1]; j = 1; }
            if (c[2] > m) { m = c[2]; j = 2; }
            if (c[3] > m) { m = c[3]; j = 3; }
            if (!(m > key)) break;
            at(t) = m;
            t = 4 * t + 1 + j;
        }
        at(t) = key;
    }
    __device__ void heapify(int n) const
    {
        for (int t = (n - 2) / 4; t >= 0; --t) sift(t, n, at(t));
    }
};

template <class K>
__host__ __device__ constexpr int heap4_groups(int kcap) { return (kcap + 2) / 4 + 1; }

// pending heap insertions per lane (a tile adds at most its masked candidates,
// so the lists are merged before a tile that could overflow one)
constexpr int kPend = 32;
static_assert(kPend >= kLeaf, "a tile can admit all of its candidates: one empty pending list must hold them");
// Defaults of the launch knobs (sidm_config; none changes a result): query
// groups of 32 / G consecutive lanes whose boxes filter the candidates,
// independent distance chains in the candidate loop, the pending count at
// which the lists are merged before a tree node's tests, and the warm-start
// bound factor (previous kernel size times it); values the autotuner picks on
// the GB300 for the 2^20 NFW halo at N_ngb = 64 (with the fixed-bound warm
// kernel: 1.47 ms per search at a bound of 1.07, 1.52 ms at 1.05)
constexpr int kGroupsDefault = 2;
// compacted candidate batches (knob knn_batch): candidates that pass the group
// filter are appended to a per-warp buffer and the distance loop runs over
// batches of kBatch of them; the buffer holds a batch's leftover (< kBatch)
// plus one whole leaf
constexpr int kBatch = 16;
constexpr int kBufCap = kBatch + kLeaf;
static_assert(kPend >= kBatch, "a batch can admit all of its candidates: one empty pending list must hold them");
constexpr int kChainsDefault = 4;
constexpr int kBatchDefault = 3;                   // 1: loop per staged leaf, 2: compacted batches, 3: 2 + fixed-bound warm kernel
constexpr int kFlushNodeDefault = 32;
constexpr float kGuessSlackDefault = 1.07f;

template <class R>
__device__ __forceinline__ float to_float_ru(R v)
{
    if constexpr (sizeof(R) == 8) return __double2float_ru((double)v);
    else return (float)v;
}

// shared memory of one warp: staged tile (shifted in place) | ids | traversal
// stack | heap groups | pending keys (the child boxes of a node live in
// registers, one per lane); 14.1 KB at N_ngb = 64 in the mixed form, so 16
// warps fit on an SM
template <class R, class K, int G, bool BATCH = false>
__host__ __device__ constexpr size_t knn_warp_bytes_t(int kcap)
{
    // the batch buffer takes the place of the staged tile and its ids
    return ((BATCH ? (size_t)kBufCap * sizeof(typename Vec4<R>::T) : TileStageT<R, false, 1>::bytes() + 32 * 4) +
            kStack * 4 + 2 * G * 16 +
            (size_t)heap4_groups<K>(kcap) * 32 * 4 * sizeof(K) + (size_t)kPend * 32 * sizeof(K) + 15) / 16 * 16;
}

static_assert((TileStageT<float, false, 1>::bytes() + 32 * 4 + kStack * 4) % 16 == 0 &&
                  (TileStageT<double, false, 1>::bytes() + 32 * 4 + kStack * 4) % 16 == 0 &&
                  (kBufCap * 16 + kStack * 4) % 16 == 0,
              "the heap groups are read as 16-byte vectors");
template <class R, bool NBR, bool TMA, int G, int CH, bool BATCH>
__global__ void k_knn(KnnParams p)
{
    static_assert(G == 2 || G == 4 || G == 8, "lane groups are 16, 8 or 4 lanes");
    static_assert(CH == 4 || CH == 8, "four or eight independent distance chains");
    static_assert(!(BATCH && TMA), "compacted batches read candidates straight into registers");
    using V = typename Vec4<R>::T;
    using K = typename KeyOf<R, NBR>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char* base = smem + wid * knn_warp_bytes_t<R, K, G, BATCH>(p.kcap);
    TileStageT<R, TMA, 1> stage(base);
    V* bufv = (V*)base;                            // BATCH: [kBufCap] candidates (w: slot, or id with NBR)
    uint32_t* tids = (uint32_t*)(base + TileStageT<R, TMA, 1>::bytes());
    int* stack = BATCH ? (int*)(base + (size_t)kBufCap * sizeof(V)) : (int*)(tids + 32);
    float4* gbox = (float4*)(stack + kStack);      // [G][2]: box lo, hi of each lane group
    K* heapg = (K*)(gbox + 2 * G);                 // 16-byte aligned: 528 + 128 + 4 kStack bytes in, + boxes
    K* pend = heapg + (size_t)heap4_groups<K>(p.kcap) * 32 * 4;   // [kPend][32]
    const Heap4<K> hp{heapg, lane};
    stage.init(lane);
    unsigned long long n_cand = 0ull, n_ins = 0ull, n_tiles_all = 0ull, n_tiles_max = 0ull, n_redo = 0ull;

    while (true) {
        int leaf = 0;
        if (lane == 0) leaf = (int)atomicAdd(p.work, 1u);
        leaf = __shfl_sync(0xffffffffu, leaf, 0);
        if (p.leaf_list) {
            if ((unsigned)leaf >= *p.list_len) break;
            leaf = p.leaf_list[leaf];
        } else if (leaf >= p.L) {
            break;
        }
        const int h = p.leaf_halo[leaf];
        const int k = p.ngb[h];
        const int leaf0 = p.leaf_off[h];
        const int nleaf = p.leaf_off[h + 1] - leaf0;
        const int64_t hb = p.halo_off[h];
        const int64_t nh = p.halo_off[h + 1] - hb;
        const int A = leaf - leaf0;
        const int countA = (int)min((int64_t)kLeaf, nh - (int64_t)A * kLeaf);
        const bool active = lane < countA;
        const HaloFrame fr = p.frame[h];
        const V q = ((const V*)p.P4)[(int64_t)leaf * kLeaf + lane];
        // a buffered candidate's w holds its slot (its id with NBR), so the query
        // recognises itself
        const uint32_t own = NBR ? (BATCH && active ? p.ID[(int64_t)leaf * kLeaf + lane] : 0u)
                                 : (uint32_t)leaf * kLeaf + lane;
        const float4 cA = p.cell[leaf];
        const float4 qlo = p.nlo[leaf], qhi = p.nhi[leaf];
        unsigned long long n_tiles = 0ull;
        bool failed = false;
        // Warm start: q.w holds the particle's kernel size of the previous call.
        // Pass 0 starts with the bound key of (h_prev * slack)^2, so only
        // candidates inside that bound enter; a lane that collects fewer than k
        // of them is redone by the cold pass 1 (Morton-window fill, unbounded
        // start).  In both passes the first k admitted keys are stored unsorted
        // and heapified once.
        const bool guess = p.use_guess && active && q.w > R(0);
        K bound_key = ~K(0);
        if (guess) {
            R r;
            if constexpr (sizeof(R) == 4) r = __fmul_ru((float)q.w, p.slack);
            else r = __dmul_ru((double)q.w, (double)p.slack);
            bound_key = make_key<R, NBR>(mul_ru(r, r), 0xFFFFFFFFu);
        }
        K result = K(0);
        bool todo = active;
        for (int pass = __any_sync(0xffffffffu, guess) ? 0 : 1; pass < 2; ++pass) {
        const bool act = pass == 0 ? guess : todo;
        if (!__any_sync(0xffffffffu, act)) break;
        hp.clear_tail(k);
        K root = (pass == 0 && act) ? bound_key : ~K(0);
        int nfill = 0, np = 0;                         // heap fill level, pending keys
        bool heaped = false;

        int nbuf = 0;                                  // BATCH: candidates in the buffer
        // merge the pending keys of every lane into its heap (each lane works
        // on its own heap column; no lane reads another's)
        auto flush = [&]() {
            if (!heaped && nfill == k) {               // the heap array is full: order it once
                hp.heapify(k);
                root = hp.at(0);
                heaped = true;
            }
            for (int i = 0; i < np; ++i) {
                const K key = pend[i * 32 + lane];
                if (key < root) {
                    ++n_ins;
                    hp.sift(0, k, key);
                    root = hp.at(0);
                }
            }
            np = 0;
        };

        float3 pq;                                     // query point in the halo frame
        if constexpr (sizeof(R) == 4) {
            pq = make_float3(__fadd_rn(cA.x, (float)q.x), __fadd_rn(cA.y, (float)q.y), __fadd_rn(cA.z, (float)q.z));
        } else {
            pq = make_float3(__double2float_rn((double)q.x - fr.O[0]), __double2float_rn((double)q.y - fr.O[1]),
                             __double2float_rn((double)q.z - fr.O[2]));
        }
        // boxes of the query points of each group of 32 / G consecutive
        // lanes (shared memory): a candidate is kept if it lies within the
        // largest bound of some group's lanes from that group's box (the union is
        // tighter than the whole leaf's box; the mask stays warp-uniform)
        constexpr int kGL = 32 / G;
        {
            float lx = active ? pq.x : INFINITY, ly = active ? pq.y : INFINITY, lz = active ? pq.z : INFINITY;
            float ux = active ? pq.x : -INFINITY, uy = active ? pq.y : -INFINITY, uz = active ? pq.z : -INFINITY;
            for (int o = kGL / 2; o > 0; o >>= 1) {
                lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
                ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
                lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
                ux = fmaxf(ux, __shfl_xor_sync(0xffffffffu, ux, o));
                uy = fmaxf(uy, __shfl_xor_sync(0xffffffffu, uy, o));
                uz = fmaxf(uz, __shfl_xor_sync(0xffffffffu, uz, o));
            }
            __syncwarp();
            if (lane % kGL == 0) {
                gbox[2 * (lane / kGL)] = make_float4(lx, ly, lz, 0.f);
                gbox[2 * (lane / kGL) + 1] = make_float4(ux, uy, uz, 0.f);
            }
            __syncwarp();
        }
        auto my_r2 = [&]() -> float {
            if (!act) return -1.0f;
            float r = to_float_ru<R>(sqrt_ru(key_d2<R, NBR>(root)));
            r = __fadd_ru(__fmul_ru(r, 1.0f + 0x1p-20f), fr.margin);
            return __fmul_ru(r, r);
        };
        // this lane's entry of candidate leaf Bl and the leaf's frame origin (the
        // plain path loads both straight into registers, so a caller can fetch
        // the next leaf early; the shift needs the origin as soon as the entry)
        struct Fetched { V c; float4 cell; };
        auto fetch = [&](int Bl) -> Fetched {
            Fetched f{};
            if constexpr (!TMA) f.c = ((const V*)p.P4)[(int64_t)(leaf0 + Bl) * kLeaf + lane];
            if constexpr (sizeof(R) == 4) f.cell = p.cell[leaf0 + Bl];
            return f;
        };
        // the largest bound of each lane group (r2g) and of all lanes (r2all),
        // from each lane's bound r2 (my_r2); an unbounded lane (its heap not yet
        // full in the cold pass) counts as infinite
        struct GroupBounds { float g[G]; float all; };
        auto group_bounds = [&](float r2, bool mine) -> GroupBounds {
            float lr2 = -1.f;
            if (act && mine) lr2 = isnan(r2) ? INFINITY : r2;
            for (int o = kGL / 2; o > 0; o >>= 1) lr2 = fmaxf(lr2, __shfl_xor_sync(0xffffffffu, lr2, o));
            GroupBounds b;
            b.all = -1.f;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                b.g[g] = __shfl_sync(0xffffffffu, lr2, g * kGL);
                b.all = fmaxf(b.all, b.g[g]);
            }
            return b;
        };
        // BATCH: the distances from every active query to the first nb buffered
        // candidates (CH independent chains), admitted like the per-leaf loop
        // below; the entries after them move to the front
        auto run_batch = [&](int nb) {
            if (__any_sync(0xffffffffu, np + nb > kPend)) flush();
            __syncwarp();
            if (act) {
                n_cand += (unsigned long long)nb;
                for (int t = 0; t < nb; t += CH) {
                    K key[CH];
                    bool ok[CH];
#pragma unroll
                    for (int u = 0; u < CH; ++u) {
                        const int idx = t + u < nb ? t + u : t;
                        const V cj = bufv[idx];
                        const uint32_t who = sizeof(R) == 4 ? __float_as_uint((float)cj.w) : (uint32_t)(double)cj.w;
                        const R dx = sub_rn(cj.x, q.x), dy = sub_rn(cj.y, q.y), dz = sub_rn(cj.z, q.z);
                        const R d2 = fma_rn(dz, dz, fma_rn(dy, dy, mul_rn(dx, dx)));
                        key[u] = make_key<R, NBR>(d2, who);
                        ok[u] = t + u < nb && who != own;
                    }
#pragma unroll
                    for (int u = 0; u < CH; ++u) {
                        if (ok[u] && key[u] < root) {
                            if (nfill < k) hp.at(nfill++) = key[u];
                            else pend[(np++) * 32 + lane] = key[u];
                        }
                    }
                }
            }
            __syncwarp();
            const int rem = nbuf - nb;                 // < 32
            V tmp{};
            if (lane < rem) tmp = bufv[nb + lane];
            __syncwarp();
            if (lane < rem) bufv[lane] = tmp;
            nbuf = rem;
            __syncwarp();
        };
        auto drain = [&]() {
            if constexpr (BATCH) { if (nbuf > 0) run_batch(nbuf); }
        };
        // mine: this lane's query reaches leaf Bl; gb: group_bounds of the lanes'
        // bounds; craw: fetch(Bl) (unused on the bulk-copy path, which stages the
        // leaf here)
        auto process = [&](int Bl, bool mine, const GroupBounds& gb, const Fetched& craw) {
            const int Bg = leaf0 + Bl;
            const int countB = (int)min((int64_t)kLeaf, nh - (int64_t)Bl * kLeaf);
            V c;
            if constexpr (TMA) c = stage.load_lane((const V*)p.P4 + (int64_t)Bg * kLeaf, lane, p.cnt);
            else c = craw.c;
            // shift the candidates into the query leaf's frame (exact shift)
            if constexpr (sizeof(R) == 4) {
                const float4 cB = craw.cell;
                c.x = __fadd_rn(c.x, __fsub_rn(cB.x, cA.x));
                c.y = __fadd_rn(c.y, __fsub_rn(cB.y, cA.y));
                c.z = __fadd_rn(c.z, __fsub_rn(cB.z, cA.z));
            }
            // candidates farther from a lane group's box than the largest bound of
            // its lanes cannot enter one of their heaps: the loops skip the
            // candidates no group can reach (an unbounded lane, before its heap is
            // full in the cold pass, keeps them all)
            const float r2all = gb.all;
            uint32_t cmask;
            if (!(r2all < INFINITY)) {
                cmask = countB == kLeaf ? 0xffffffffu : ((1u << countB) - 1u);
            } else {
                float3 pc;                             // candidate in the halo frame
                if constexpr (sizeof(R) == 4) {
                    pc = make_float3(__fadd_rn(cA.x, c.x), __fadd_rn(cA.y, c.y), __fadd_rn(cA.z, c.z));
                } else {
                    pc = make_float3(__double2float_rn((double)c.x - fr.O[0]), __double2float_rn((double)c.y - fr.O[1]),
                                     __double2float_rn((double)c.z - fr.O[2]));
                }
                bool reach = false;
#pragma unroll
                for (int g = 0; g < G; ++g)
                    reach = reach || (gb.g[g] >= 0.f && point_gap2_rd(pc, gbox[2 * g], gbox[2 * g + 1]) <= gb.g[g]);
                cmask = __ballot_sync(0xffffffffu, lane < countB && reach);
            }
            ++n_tiles;
            if (cmask == 0u) return;                   // no candidate of this leaf can enter
            if constexpr (BATCH) {
                // append the candidates that pass to the buffer, in lane order
                if ((cmask >> lane) & 1u) {
                    V e = c;
                    const uint32_t who = NBR ? p.ID[(int64_t)Bg * kLeaf + lane] : (uint32_t)Bg * kLeaf + lane;
                    if constexpr (sizeof(R) == 4) e.w = __uint_as_float(who); else e.w = (R)who;
                    bufv[nbuf + __popc(cmask & ((1u << lane) - 1u))] = e;
                }
                nbuf += __popc(cmask);
                __syncwarp();
                while (nbuf >= kBatch) run_batch(kBatch);
                return;
            }
            // room for this tile's candidates in every pending list
            if (__any_sync(0xffffffffu, np + __popc(cmask) > kPend)) flush();
            __syncwarp();
            V* sh = stage.shifted();
            sh[lane] = c;
            if (NBR) tids[lane] = p.ID[(int64_t)Bg * kLeaf + lane];
            __syncwarp();
            if (act && mine) {
                n_cand += (unsigned long long)__popc(cmask);
                // the masked candidates CH at a time (independent distance
                // chains); an admitted key fills the heap array (unsorted, heapified
                // at the next merge) until it holds k keys, then waits in the
                // pending list, for which room was made before the tile
                for (uint32_t mm = cmask; mm;) {
                    int t[CH];
#pragma unroll
                    for (int u = 0; u < CH; ++u) { t[u] = __ffs(mm) - 1; mm &= mm - 1u; }   // -1: none left
                    K key[CH];
#pragma unroll
                    for (int u = 0; u < CH; ++u) {
                        const V cj = sh[t[u] >= 0 ? t[u] : t[0]];
                        const R dx = sub_rn(cj.x, q.x), dy = sub_rn(cj.y, q.y), dz = sub_rn(cj.z, q.z);
                        const R d2 = fma_rn(dz, dz, fma_rn(dy, dy, mul_rn(dx, dx)));
                        key[u] = make_key<R, NBR>(d2, NBR ? tids[t[u] >= 0 ? t[u] : t[0]] : 0u);
                    }
#pragma unroll
                    for (int u = 0; u < CH; ++u) {
                        if (t[u] >= 0 && key[u] < root && !(Bl == A && t[u] == lane)) {
                            if (nfill < k) hp.at(nfill++) = key[u];
                            else pend[(np++) * 32 + lane] = key[u];
                        }
                    }
                }
            }
            __syncwarp();
        };

        // 1) cold pass: Morton-window leaves around A holding at least k+1 particles
        int wlo = 0, whi = -1;
        if (pass == 1) {
            wlo = A; whi = A;
            int64_t wcount = countA;
            while (wcount < k + 1 && (wlo > 0 || whi < nleaf - 1)) {
                if (whi < nleaf - 1) { ++whi; wcount += min((int64_t)kLeaf, nh - (int64_t)whi * kLeaf); }
                if (wcount < k + 1 && wlo > 0) { --wlo; wcount += kLeaf; }
            }
            // the window holds at least k other particles, so every lane's heap is
            // full after it: order it and merge the window's keys beyond the first k
            for (int Bl = wlo; Bl <= whi; ++Bl) process(Bl, true, group_bounds(my_r2(), true), fetch(Bl));
            drain();
            flush();
        }

        // 2) tree walk.  A node is visited iff the query point of some lane lies
        //    within that lane's current k-th distance (+ margin) of the node's box;
        //    accepted leaves are processed at once so the bound keeps shrinking.
        // the boxes of the children being tested, one per lane, in registers
        float4 clo = make_float4(0.f, 0.f, 0.f, 0.f), chi = clo;
        auto load_boxes = [&](int g0, int n) {
            if (lane < n) { clo = p.nlo[g0 + lane]; chi = p.nhi[g0 + lane]; }
        };
        // this lane's query within r2 of child c's box (every lane takes part)
        auto near_child = [&](int c, float r2) -> bool {
            const float4 lo = make_float4(__shfl_sync(0xffffffffu, clo.x, c), __shfl_sync(0xffffffffu, clo.y, c),
                                          __shfl_sync(0xffffffffu, clo.z, c), 0.f);
            const float4 hi = make_float4(__shfl_sync(0xffffffffu, chi.x, c), __shfl_sync(0xffffffffu, chi.y, c),
                                          __shfl_sync(0xffffffffu, chi.z, c), 0.f);
            return r2 >= 0.f && point_gap2_rd(pq, lo, hi) <= r2;
        };
        // bit c: the query of some lane lies within its bound of box c; the
        // lane's own bits and bound are kept for the leaves of this node.
        // Every query point lies in the query leaf's box, so a child farther
        // from that box than the largest lane bound is out of reach of every
        // lane: one box test per child (a lane each) leaves the per-lane
        // point tests to the children that pass it.
        uint32_t lane_bits = 0u;
        float node_r2 = -1.0f;
        auto accept = [&](int n, float r2, uint32_t skip) -> uint32_t {
            float r2max = r2;
            for (int o = 16; o > 0; o >>= 1) r2max = fmaxf(r2max, __shfl_xor_sync(0xffffffffu, r2max, o));
            const uint32_t near =
                __ballot_sync(0xffffffffu, lane < n && box_gap2_rd(qlo, qhi, clo, chi) <= r2max) & ~skip;
            uint32_t bits = 0u;
            for (uint32_t m = near; m; m &= m - 1u) {
                const int c = __ffs(m) - 1;
                if (near_child(c, r2)) bits |= 1u << c;
            }
            lane_bits = bits;
            node_r2 = r2;
            return __reduce_or_sync(0xffffffffu, bits);
        };
        // leaves of the Morton window among local leaves first .. first+n-1
        auto window_mask = [&](int first, int n) -> uint32_t {
            const int lo = max(wlo - first, 0), hi = min(whi - first, n - 1);
            if (lo > hi) return 0u;
            return ((2u << hi) - 1u) & ~((1u << lo) - 1u);
        };
        // the warm pass's bound barely moves, so a leaf reuses the lane's node test
        // (a larger, older bound only admits more); the cold pass re-tests with the
        // bound its nearer leaves have shrunk
        auto visit_leaf = [&](int Bl, int c) {
            const float r2 = my_r2();
            const bool mine = near_child(c, r2);
            if (__any_sync(0xffffffffu, mine)) process(Bl, mine, group_bounds(r2, mine), fetch(Bl));
        };
        // Accepted children are visited nearest first (box gap to the query leaf),
        // so the k-th bound shrinks early.  rank = position among the accepted.
        auto order_rank = [&](uint32_t acc, int n) -> int {
            const bool mine_acc = lane < n && ((acc >> lane) & 1u);
            const float pr = mine_acc ? box_gap2_rd(qlo, qhi, clo, chi) : INFINITY;
            int rank = 0;
            for (int j = 0; j < n; ++j) {
                const float pj = __shfl_sync(0xffffffffu, pr, j);
                if ((acc >> j) & 1u) rank += (pj < pr || (pj == pr && j < lane)) ? 1 : 0;
            }
            return rank;
        };
        // the warm pass starts from a tight bound, so it takes the accepted
        // children in index order; the cold pass visits the nearest first
        auto visit_leaves_in_order = [&](uint32_t acc, int n, int first_local) {
            if (acc == 0u) return;
            if (pass == 0) {
                // index order; the next accepted leaf is fetched before this one is
                // processed, so its load overlaps this leaf's candidate loop.  Every
                // leaf of the node reuses the lanes' node-test bounds, so the group
                // bounds of a lane set are formed once per node (a lane whose query
                // misses a leaf only widens the mask, never narrows it)
                uint32_t m = acc;
                int c = __ffs(m) - 1;
                m &= m - 1u;
                Fetched cur = fetch(first_local + c);
                const GroupBounds gb = group_bounds(node_r2, lane_bits != 0u);
                while (true) {
                    const int cn = __ffs(m) - 1;       // -1: none left
                    m &= m - 1u;
                    Fetched nxt{};
                    if (cn >= 0) nxt = fetch(first_local + cn);
                    const bool mine = (lane_bits >> c) & 1u;
                    if (__any_sync(0xffffffffu, mine)) process(first_local + c, mine, gb, cur);
                    if (cn < 0) break;
                    c = cn;
                    cur = nxt;
                }
                return;
            }
            const int rank = order_rank(acc, n);
            const int cnt = __popc(acc);
            for (int r = 0; r < cnt; ++r) {
                const uint32_t m = __ballot_sync(0xffffffffu, lane < n && ((acc >> lane) & 1u) && rank == r);
                const int c = __ffs(m) - 1;
                visit_leaf(first_local + c, c);
            }
        };
        auto push_in_order = [&](uint32_t acc, int n, int lev, int first_local, int& sp) -> bool {
            const int rank = pass == 0 ? __popc(acc & ((1u << lane) - 1u)) : order_rank(acc, n);
            const int cnt = __popc(acc);
            if (sp + cnt > kStack) return false;
            if (lane < n && ((acc >> lane) & 1u)) stack[sp + cnt - 1 - rank] = (lev << 24) | (first_local + lane);
            sp += cnt;
            __syncwarp();
            return true;
        };
        const int top = p.top[h];
        const int32_t* loff = p.lvl_off;
        const int Hp = p.H + 1;
        int sp = 0;
        {
            const int nb = loff[top * Hp + h];
            const int ntop = loff[top * Hp + h + 1] - nb;   // at most kArity
            load_boxes(nb, ntop);
            const uint32_t acc = accept(ntop, my_r2(), top == 0 ? window_mask(0, ntop) : 0u);
            if (top == 0) visit_leaves_in_order(acc, ntop, 0);
            else if (!push_in_order(acc, ntop, top, 0, sp)) failed = true;
        }
        while (sp > 0 && !failed) {
            const int e = stack[--sp];
            __syncwarp();
            const int lev = e >> 24, idx = e & 0xFFFFFF;
            const int cl = lev - 1;
            const int cb = loff[cl * Hp + h];
            const int cc = loff[cl * Hp + h + 1] - cb;
            const int first = idx * kArity;
            const int nch = min(kArity, cc - first);
            // tighten the bounds before the node tests once enough keys wait
            if (__any_sync(0xffffffffu, np >= p.flush_node)) flush();
            load_boxes(cb + first, nch);
            const uint32_t acc = accept(nch, my_r2(), cl == 0 ? window_mask(first, nch) : 0u);
            if (cl == 0) visit_leaves_in_order(acc, nch, first);
            else if (!push_in_order(acc, nch, cl, first, sp)) failed = true;
        }
        drain();
        flush();
        if (act && heaped) { result = root; todo = false; }
        if (pass == 0 && act && todo) ++n_redo;
        }   // passes
        if (failed && lane == 0) raise_status(p.cnt, SIDM_DEV_STACK);
        n_tiles_all += n_tiles;
        n_tiles_max = n_tiles > n_tiles_max ? n_tiles : n_tiles_max;

        // 3) outputs
        if (active) {
            const int64_t u = hb + (int64_t)A * kLeaf + lane;
            const R hval = sqrt_rn(key_d2<R, NBR>(result));
            if (p.h_out) {
                ((R*)p.h_out)[u] = hval;
                ((R*)((V*)p.P4 + (int64_t)leaf * kLeaf + lane))[3] = hval;
                if (p.hprev) ((R*)p.hprev)[u] = hval;
            }
            if constexpr (NBR) {
                // heap sort: repeatedly move the maximum behind the shrinking heap
                for (int end = k - 1; end > 0; --end) {
                    const K top_key = hp.at(0);
                    const K last = hp.at(end);
                    hp.at(end) = top_key;
                    hp.sift_masked(0, end, last);
                }
                for (int t = 0; t < k; ++t) p.nbr[u * p.k_stride + t] = (uint32_t)(hp.at(t) & 0xFFFFFFFFull);
            }
        }
        __syncwarp();
    }
    // diagnostics: tiles, lane-level candidates, heap insertions, worst leaf
    for (int o = 16; o > 0; o >>= 1) {
        n_cand += __shfl_xor_sync(0xffffffffu, n_cand, o);
        n_ins += __shfl_xor_sync(0xffffffffu, n_ins, o);
        n_redo += __shfl_xor_sync(0xffffffffu, n_redo, o);
    }
    if (lane == 0) {
        atomicAdd(&p.cnt->diag[0], n_tiles_all);
        atomicAdd(&p.cnt->diag[1], n_cand);
        atomicAdd(&p.cnt->diag[2], n_ins);
        atomicMax(&p.cnt->diag[3], n_tiles_max);
        if (n_redo) atomicAdd(&p.cnt->diag[7], n_redo);
    }
    stage.finish(lane, p.cnt);
}

// ---------------------------------------------------------------------------
// Warm-started search.  From the second call on every particle carries its
// previous kernel size, and only candidates inside slack x h_prev are admitted
// (reading C14).  That bound is fixed for the whole query leaf, so:
//  * the tree is walked level by level (the child boxes of the next frontier
//    node load while the current one is tested); each child's box is tested
//    against the boxes of the walk's lane groups, each grown by the largest
//    bound of its lanes (one box test per child and group, no per-lane point
//    tests), and the accepted leaves are listed;
//  * the listed leaves are loaded two ahead; a candidate is kept if it lies
//    within some filter group's largest bound of that group's box, a test made
//    in the query leaf's own frame with directed rounding, where the box gap is
//    a lower bound of the canonical distance (no margin needed); kept
//    candidates go to a per-warp ring;
//  * full batches of kWBatch ring entries are tested against all 32 queries
//    with branch-free admission: a lane stores every key at its next free slot
//    and advances the slot only when the key is below its bound;
//  * the query leaf's own particles are tested first, with the exclusion of
//    the query itself, so the batch loop needs none.
// The keys of a lane sit in shared memory as [slot][lane]: slots 0..k-1 are a
// 4-ary max-heap (filled unsorted, heapified once), slots k..k+2 stay zero (the
// missing children of the last nodes), and up to kWPend further keys wait
// there until a merge.  A leaf goes to a list that the per-lane search (k_knn,
// warm-started, failing lanes cold) then redoes when a lane admits fewer than k
// keys (its guess was too small), when a group box is much wider than its
// bound (see kSpreadWalk), or when the walk's frontier overflows; so the result
// is the same exact k-th distance as a cold search.
constexpr int kWRing = 40;      // candidate ring entries
constexpr int kWBatch = 8;      // candidates per batch (batches start at multiples of it: never wrap)
constexpr int kWList = 64;      // accepted leaves listed before they are streamed
constexpr int kWStack = 128;    // two frontier buffers of the walk, 64 nodes each (an overflow
                                // hands the leaf to the redo)
constexpr int kWPad = 3;        // zero slots after the heap
constexpr int kWPend = 32;      // keys a lane may hold beyond k before a merge (room enough that
                                // merges are rare and most lanes order their heaps together)
static_assert(kWRing % kWBatch == 0 && kWRing >= kWBatch - 1 + kLeaf, "the ring holds a batch's leftover plus a leaf");
static_assert(kWPend >= kWBatch, "one batch fits after a merge");
constexpr int kWarmMaxWarps = 8;   // the kernel's launch bound: 256 threads, two CTAs per SM
constexpr int kWalkGroups = 4;     // lane groups of the tree walk (8 lanes each)
// a leaf goes to the per-lane search when the box of a walk group is wider than
// kSpreadWalk times its largest bound, or a filter group's than kSpreadFilter times
constexpr float kSpreadWalk = 3.0f;
constexpr float kSpreadFilter = 4.0f;

template <class R, class K, int G>
__host__ __device__ constexpr size_t warm_warp_bytes(int kcap)
{
    return ((size_t)kWRing * sizeof(typename Vec4<R>::T) + (size_t)(kWList + kWStack) * 4 + (size_t)2 * kWalkGroups * 16 +
            (size_t)(kcap + kWPad + kWPend) * 32 * sizeof(K) + 15) / 16 * 16;
}

template <class R, int G>
__global__ void __launch_bounds__(kWarmMaxWarps * 32, 2) k_knn_warm(KnnParams p, int32_t* redo_list, unsigned int* redo_len)
{
    static_assert(G == 2 || G == 4, "lane groups of 16 or 8 lanes");
    using V = typename Vec4<R>::T;
    using K = typename KeyOf<R, false>::T;
    constexpr bool kF32 = sizeof(R) == 4;
    constexpr int kGL = 32 / G;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char* base = smem + wid * warm_warp_bytes<R, K, G>(p.kcap);
    V* ring = (V*)base;
    int* list = (int*)(base + (size_t)kWRing * sizeof(V));
    int* fbuf = list + kWList;                         // [2][kWStack / 2] frontier buffers of the walk
    float4* wbox = (float4*)(fbuf + kWStack);          // [kWalkGroups][2]: walk group boxes (halo frame), lo.w = bound
    K* keys = (K*)(wbox + 2 * kWalkGroups);            // [kcap + kWPad + kWPend][32]
    const uint32_t lt = (1u << lane) - 1u;
    const int Hp = p.H + 1;
    // the lanes redone cold are counted by the per-lane search that redoes them
    unsigned long long n_cand = 0ull, n_ins = 0ull, n_tiles = 0ull, n_tiles_max = 0ull;

    while (true) {
        int leaf = 0;
        if (lane == 0) leaf = (int)atomicAdd(p.work, 1u);
        leaf = __shfl_sync(FULL, leaf, 0);
        if (leaf >= p.L) break;
        const int h = p.leaf_halo[leaf];
        const int k = p.ngb[h];
        const int leaf0 = p.leaf_off[h];
        const int64_t hb = p.halo_off[h];
        const int64_t nh = p.halo_off[h + 1] - hb;
        const int A = leaf - leaf0;
        const int countA = (int)min((int64_t)kLeaf, nh - (int64_t)A * kLeaf);
        const bool active = lane < countA;
        const V q = ((const V*)p.P4)[(int64_t)leaf * kLeaf + lane];
        const unsigned long long tiles0 = n_tiles;
        // a particle without a previous kernel size sends its leaf to the redo
        if (__any_sync(FULL, active && !(q.w > R(0)))) {
            if (lane == 0) { const unsigned r = atomicAdd(redo_len, 1u); redo_list[r] = leaf; }
            continue;
        }
        const HaloFrame fr = p.frame[h];
        const float4 cA = p.cell[leaf];
        // the lane's bound key: (slack h_prev)^2 rounded up; inactive lanes admit nothing
        K root = K(0);
        float r2walk = -1.0f;                          // the walk's bound in the halo frame (with the margin)
        if (active) {
            R r;
            if constexpr (kF32) r = __fmul_ru((float)q.w, p.slack);
            else r = __dmul_ru((double)q.w, (double)p.slack);
            const R b2 = mul_ru(r, r);
            root = make_key<R, false>(b2, 0u);
            float rf = to_float_ru<R>(sqrt_ru(b2));
            rf = __fadd_ru(__fmul_ru(rf, 1.0f + 0x1p-20f), fr.margin);
            r2walk = __fmul_ru(rf, rf);
        }
        // group boxes: the walk's in the halo frame (the frame of the node
        // boxes), the candidate filter's in the query leaf's frame (mixed form;
        // the FP64 form filters in the halo frame, with the walk's bounds)
        float3 pq;
        if constexpr (kF32) {
            pq = make_float3(__fadd_rn(cA.x, (float)q.x), __fadd_rn(cA.y, (float)q.y), __fadd_rn(cA.z, (float)q.z));
        } else {
            pq = make_float3(__double2float_rn((double)q.x - fr.O[0]), __double2float_rn((double)q.y - fr.O[1]),
                             __double2float_rn((double)q.z - fr.O[2]));
        }
        // walk boxes: groups of 8 lanes (a large bound of one lane grows only its
        // own group's box); the bound of each group is stored in its lo.w.  On the
        // halo's sparse outer shell a few consecutive particles of the Morton
        // curve can lie on opposite sides of the halo: a group box much wider
        // than its bound would accept most of the halo, so such a leaf is left
        // to the per-lane search (the redo list, warm-started)
        bool spread = false;
        {
            constexpr int kWL = 32 / kWalkGroups;
            float v[7] = {active ? pq.x : INFINITY, active ? pq.y : INFINITY, active ? pq.z : INFINITY,
                          active ? -pq.x : INFINITY, active ? -pq.y : INFINITY, active ? -pq.z : INFINITY, -r2walk};
#pragma unroll
            for (int o = kWL / 2; o > 0; o >>= 1) {
#pragma unroll
                for (int i = 0; i < 7; ++i) v[i] = fminf(v[i], __shfl_xor_sync(FULL, v[i], o));
            }
            if (lane % kWL == 0) {
                wbox[2 * (lane / kWL)] = make_float4(v[0], v[1], v[2], -v[6]);
                wbox[2 * (lane / kWL) + 1] = make_float4(-v[3], -v[4], -v[5], 0.f);
                const float ext = fmaxf(fmaxf(-v[3] - v[0], -v[4] - v[1]), -v[5] - v[2]);
                spread = -v[6] >= 0.f && ext * ext > kSpreadWalk * kSpreadWalk * -v[6];
            }
            __syncwarp();
        }
        // filter boxes: groups of 32 / G lanes, in the query leaf's frame (mixed
        // form) or the halo frame (FP64 form, with the walk's bounds)
        float r2f[G];
        float4 flo[G], fhi[G];
        {
            float v[6];
            if constexpr (kF32) {
                v[0] = active ? (float)q.x : INFINITY;  v[1] = active ? (float)q.y : INFINITY;  v[2] = active ? (float)q.z : INFINITY;
                v[3] = active ? -(float)q.x : INFINITY; v[4] = active ? -(float)q.y : INFINITY; v[5] = active ? -(float)q.z : INFINITY;
            } else {
                v[0] = active ? pq.x : INFINITY;  v[1] = active ? pq.y : INFINITY;  v[2] = active ? pq.z : INFINITY;
                v[3] = active ? -pq.x : INFINITY; v[4] = active ? -pq.y : INFINITY; v[5] = active ? -pq.z : INFINITY;
            }
#pragma unroll
            for (int o = kGL / 2; o > 0; o >>= 1) {
#pragma unroll
                for (int i = 0; i < 6; ++i) v[i] = fminf(v[i], __shfl_xor_sync(FULL, v[i], o));
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                flo[g] = make_float4(__shfl_sync(FULL, v[0], g * kGL), __shfl_sync(FULL, v[1], g * kGL),
                                     __shfl_sync(FULL, v[2], g * kGL), 0.f);
                fhi[g] = make_float4(-__shfl_sync(FULL, v[3], g * kGL), -__shfl_sync(FULL, v[4], g * kGL),
                                     -__shfl_sync(FULL, v[5], g * kGL), 0.f);
            }
        }
        // the filter's bounds: the largest bound key of each group (mixed: the
        // exact bound; FP64: the walk's, with the margin)
        auto filter_bounds = [&]() {
            float b = -1.0f;
            if constexpr (kF32) { if (active) b = key_d2<R, false>(root); }
            else b = r2walk;
#pragma unroll
            for (int o = kGL / 2; o > 0; o >>= 1) b = fmaxf(b, __shfl_xor_sync(FULL, b, o));
#pragma unroll
            for (int g = 0; g < G; ++g) r2f[g] = __shfl_sync(FULL, b, g * kGL);
        };
        filter_bounds();
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const float ext = fmaxf(fmaxf(fhi[g].x - flo[g].x, fhi[g].y - flo[g].y), fhi[g].z - flo[g].z);
            spread = spread || (r2f[g] >= 0.f && ext * ext > kSpreadFilter * kSpreadFilter * r2f[g]);
        }
        if (__any_sync(FULL, spread)) {
            if (lane == 0) { const unsigned r = atomicAdd(redo_len, 1u); redo_list[r] = leaf; }
            continue;
        }
        // zero the slots after the heap of this leaf's k
        for (int i = 0; i < kWPad; ++i) keys[(k + i) * 32 + lane] = K(0);

        int cnt = 0;                                   // keys held (slots 0..k-1, then k+3..)
        bool heaped = false;
        auto sift = [&](int t, K key) {
            while (true) {
                const int c0 = 4 * t + 1;
                if (c0 >= k) break;
                const K* cp = keys + (size_t)c0 * 32 + lane;
                K m = cp[0];
                int j = 0;
                const K c1 = cp[32], c2 = cp[64], c3 = cp[96];
                if (c1 > m) { m = c1; j = 1; }
                if (c2 > m) { m = c2; j = 2; }
                if (c3 > m) { m = c3; j = 3; }
                if (!(m > key)) break;
                keys[t * 32 + lane] = m;
                t = c0 + j;
            }
            keys[t * 32 + lane] = key;
        };
        // merge the waiting keys into the heap (each lane its own column)
        auto flush = [&]() {
            if (active && cnt >= k) {
                if (!heaped) {
                    for (int t = (k - 2) / 4; t >= 0; --t) sift(t, keys[t * 32 + lane]);
                    heaped = true;
                    root = keys[lane];
                }
                for (int i = k; i < cnt; ++i) {
                    const K key = keys[(i + kWPad) * 32 + lane];
                    if (key < root) {
                        ++n_ins;
                        sift(0, key);
                        root = keys[lane];
                    }
                }
                cnt = k;
            }
            filter_bounds();
        };
        // distances from every query to the kWBatch entries at src
        auto batch = [&](const V* src, bool self) {
            if (__any_sync(FULL, cnt > k + kWPend - kWBatch)) flush();
            __syncwarp();
#pragma unroll
            for (int t = 0; t < kWBatch; t += 4) {
                K key[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const V cj = src[t + u];
                    const R dx = sub_rn(cj.x, q.x), dy = sub_rn(cj.y, q.y), dz = sub_rn(cj.z, q.z);
                    key[u] = make_key<R, false>(fma_rn(dz, dz, fma_rn(dy, dy, mul_rn(dx, dx))), 0u);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool adm = key[u] < root && !(self && t + u == (lane & (kWBatch - 1)));
                    const int slot = cnt < k ? cnt : cnt + kWPad;
                    keys[slot * 32 + lane] = key[u];
                    cnt += adm ? 1 : 0;
                }
            }
            __syncwarp();
        };
        V far;
        far.x = R(INFINITY); far.y = R(INFINITY); far.z = R(INFINITY); far.w = R(0);

        // 1) the query leaf's own particles, two batches of 16 (lanes past the
        //    leaf's end read as infinitely far)
        ring[lane] = active ? q : far;
        __syncwarp();
        if (active) n_cand += (unsigned long long)countA;
#pragma unroll
        for (int b = 0; b < kLeaf; b += kWBatch) batch(ring + b, (lane & ~(kWBatch - 1)) == b);
        __syncwarp();

        // 2) stream listed leaves: filter, append to the ring, run full batches
        int head = 0, tail = 0, navail = 0;
        auto wrap = [](int i) { return i >= kWRing ? i - kWRing : i; };   // i < 2 kWRing
        auto stage_leaf = [&](int Bl, V c, float4 cB) {
            const int countB = (int)min((int64_t)kLeaf, nh - (int64_t)Bl * kLeaf);
            bool reach = false;
            if constexpr (kF32) {
                c.x = __fadd_rn(c.x, __fsub_rn(cB.x, cA.x));     // exact shift into the query leaf's frame
                c.y = __fadd_rn(c.y, __fsub_rn(cB.y, cA.y));
                c.z = __fadd_rn(c.z, __fsub_rn(cB.z, cA.z));
                const float3 pc = make_float3(c.x, c.y, c.z);
#pragma unroll
                for (int g = 0; g < G; ++g) reach = reach || point_gap2_rd(pc, flo[g], fhi[g]) <= r2f[g];
            } else {
                const float3 pc = make_float3(__double2float_rn((double)c.x - fr.O[0]),
                                              __double2float_rn((double)c.y - fr.O[1]),
                                              __double2float_rn((double)c.z - fr.O[2]));
#pragma unroll
                for (int g = 0; g < G; ++g) reach = reach || point_gap2_rd(pc, flo[g], fhi[g]) <= r2f[g];
            }
            const uint32_t m = __ballot_sync(FULL, lane < countB && reach);
            ++n_tiles;
            if (m == 0u) return;
            if ((m >> lane) & 1u) ring[wrap(tail + __popc(m & lt))] = c;
            const int nm = __popc(m);
            tail = wrap(tail + nm);
            navail += nm;
            __syncwarp();
            while (navail >= kWBatch) {
                if (active) n_cand += (unsigned long long)kWBatch;
                batch(ring + head, false);
                head = wrap(head + kWBatch);
                navail -= kWBatch;
            }
        };
        int nl = 0;
        auto stream_list = [&]() {
            using CellT = float4;
            V c0{}, c1{};
            CellT b0{}, b1{};
            auto fetch = [&](int i, V& c, CellT& b) {
                const int Bl = list[i];
                c = ((const V*)p.P4)[(int64_t)(leaf0 + Bl) * kLeaf + lane];
                if constexpr (kF32) b = p.cell[leaf0 + Bl];
            };
            if (nl > 0) fetch(0, c0, b0);
            if (nl > 1) fetch(1, c1, b1);
            for (int i = 0; i < nl; ++i) {
                V c2{};
                CellT b2{};
                if (i + 2 < nl) fetch(i + 2, c2, b2);
                stage_leaf(list[i], c0, b0);
                c0 = c1; b0 = b1; c1 = c2; b1 = b2;
            }
            nl = 0;
            __syncwarp();
        };
        // tree walk, level by level: the accepted nodes of a level form the
        // frontier of the next; the child boxes of the next frontier node are
        // loaded while the current node's children are tested (one child per
        // lane, against every walk group's box grown by its bound)
        auto accept = [&](int n, float4 clo, float4 chi) -> uint32_t {
            bool ok = false;
            if (lane < n) {
#pragma unroll
                for (int g = 0; g < kWalkGroups; ++g) {
                    const float4 lo = wbox[2 * g];
                    ok = ok || box_gap2_rd(lo, wbox[2 * g + 1], clo, chi) <= lo.w;
                }
            }
            return __ballot_sync(FULL, ok);
        };
        auto add_leaves = [&](uint32_t acc, int first) {
            if (nl + __popc(acc) > kWList) stream_list();
            if ((acc >> lane) & 1u) list[nl + __popc(acc & lt)] = first + lane;
            nl += __popc(acc);
            __syncwarp();
        };
        bool overflow = false;
        constexpr int kWFront = kWStack / 2;
        int* front = fbuf;
        int* nextf = fbuf + kWFront;
        int nf = 0;
        const int top = p.top[h];
        const int32_t* loff = p.lvl_off;
        {
            const int nb0 = loff[top * Hp + h];
            const int ntop = loff[top * Hp + h + 1] - nb0;
            float4 clo = make_float4(0.f, 0.f, 0.f, 0.f), chi = clo;
            if (lane < ntop) { clo = p.nlo[nb0 + lane]; chi = p.nhi[nb0 + lane]; }
            const uint32_t acc = accept(ntop, clo, chi);
            if (top == 0) {
                add_leaves(acc & ~(1u << A), 0);
            } else {
                if ((acc >> lane) & 1u) front[__popc(acc & lt)] = lane;
                nf = __popc(acc);
                __syncwarp();
            }
        }
        for (int lev = top; lev > 0 && nf > 0 && !overflow; --lev) {
            const int cl = lev - 1;
            const int cb = loff[cl * Hp + h];
            const int cc = loff[cl * Hp + h + 1] - cb;
            int nn = 0;
            float4 lo0 = make_float4(0.f, 0.f, 0.f, 0.f), hi0 = lo0;
            auto load = [&](int i, float4& lo, float4& hi) {
                const int first = front[i] * kArity;
                if (lane < min(kArity, cc - first)) { lo = p.nlo[cb + first + lane]; hi = p.nhi[cb + first + lane]; }
            };
            load(0, lo0, hi0);
            for (int i = 0; i < nf; ++i) {
                float4 lo1 = make_float4(0.f, 0.f, 0.f, 0.f), hi1 = lo1;
                if (i + 1 < nf) load(i + 1, lo1, hi1);
                const int first = front[i] * kArity;
                const int nch = min(kArity, cc - first);
                uint32_t acc = accept(nch, lo0, hi0);
                if (cl == 0) {
                    if (A >= first && A < first + nch) acc &= ~(1u << (A - first));
                    add_leaves(acc, first);
                } else {
                    const int na = __popc(acc);
                    if (nn + na > kWFront) { overflow = true; break; }
                    if ((acc >> lane) & 1u) nextf[nn + __popc(acc & lt)] = first + lane;
                    nn += na;
                }
                lo0 = lo1; hi0 = hi1;
            }
            __syncwarp();
            int* t = front; front = nextf; nextf = t;
            nf = nn;
        }
        stream_list();
        // the last, partial batch: pad it with infinitely far entries
        if (navail > 0) {
            if (lane < kWBatch - navail) ring[wrap(tail + lane)] = far;
            __syncwarp();
            if (active) n_cand += (unsigned long long)navail;
            batch(ring + head, false);
        }
        flush();
        const bool ok = !active || heaped;
        if (overflow || !__all_sync(FULL, ok)) {
            if (lane == 0) { const unsigned r = atomicAdd(redo_len, 1u); redo_list[r] = leaf; }
        } else if (active) {
            const int64_t u = hb + (int64_t)A * kLeaf + lane;
            const R hval = sqrt_rn(key_d2<R, false>(root));
            ((R*)p.h_out)[u] = hval;
            ((R*)((V*)p.P4 + (int64_t)leaf * kLeaf + lane))[3] = hval;
            if (p.hprev) ((R*)p.hprev)[u] = hval;
        }
        n_tiles_max = n_tiles - tiles0 > n_tiles_max ? n_tiles - tiles0 : n_tiles_max;
        __syncwarp();
    }
    for (int o = 16; o > 0; o >>= 1) {
        n_cand += __shfl_xor_sync(FULL, n_cand, o);
        n_ins += __shfl_xor_sync(FULL, n_ins, o);
    }
    if (lane == 0) {
        atomicAdd(&p.cnt->diag[0], n_tiles);
        atomicAdd(&p.cnt->diag[1], n_cand);
        atomicAdd(&p.cnt->diag[2], n_ins);
        atomicMax(&p.cnt->diag[3], n_tiles_max);
    }
}

void fill_params(sidm_ctx* c, KnnParams& p, void* h_out, uint32_t* nbr, int k_stride, bool use_guess)
{
    const LayoutHost& L = c->lay;
    p.H = L.H; p.L = L.L;
    p.leaf_halo = c->d_leaf_halo; p.leaf_off = c->d_leaf_off; p.halo_off = c->d_halo_off;
    p.lvl_off = c->d_lvl_off; p.top = c->d_top; p.ngb = c->d_ngb; p.frame = c->d_frame;
    p.cell = c->d_cell; p.nlo = c->d_nlo; p.nhi = c->d_nhi; p.P4 = c->d_P4; p.ID = c->d_ID;
    p.h_out = h_out; p.nbr = nbr; p.k_stride = k_stride; p.kcap = c->kmax_cur; p.cnt = c->d_cnt;
    p.work = &c->d_cnt->work[0];
    p.leaf_list = nullptr; p.list_len = nullptr;
    p.hprev = nbr ? nullptr : c->d_hprev;
    p.use_guess = use_guess ? 1 : 0;
    p.slack = c->cfg.knn_slack > 0.f ? c->cfg.knn_slack : kGuessSlackDefault;
    p.flush_node = c->cfg.knn_flush > 0 ? c->cfg.knn_flush : kFlushNodeDefault;
}

// warps per CTA: at most the configured number, and of those the one with the
// most resident warps per SM (with large N_ngb the per-warp heaps make two
// small CTAs hold more warps than one large one); a CTA may use at most 227 KB
// of shared memory.  Also the persistent grid.
int pick_shape(sidm_ctx* c, const void* kern, size_t per_warp, int* warps_out, int* grid_out, int max_warps = 16)
{
    int warps = 0, occ = 0;
    for (int w = std::min(c->knn_warps, max_warps); w >= 1; --w) {
        if ((size_t)w * per_warp > (size_t)227 * 1024) continue;
        int o = 0;
        const int rc = occupancy(c, kern, w * 32, (size_t)w * per_warp, &o);
        if (rc) return rc;
        if (o * w > occ * warps) { warps = w; occ = o; }
    }
    if (warps < 1 || occ < 1) return set_err(c, SIDM_ECAPACITY, "knn kernel does not fit on an SM (ngb_max too large)");
    int grid = c->cfg.grid_ctas > 0 ? c->cfg.grid_ctas : c->sm_count * occ;
    grid = std::max(1, std::min(grid, (c->lay.L + warps - 1) / warps));
    *warps_out = warps;
    *grid_out = grid;
    return SIDM_OK;
}

// redo: the leaves the fixed-bound warm kernel listed (their count and the
// work counter were zeroed before it ran)
template <class R, bool NBR, bool TMA, int G, int CH, bool BATCH = false>
int launch_t(sidm_ctx* c, void* h_out, uint32_t* nbr, int k_stride, bool use_guess, cudaStream_t s, bool redo = false)
{
    using K = typename KeyOf<R, NBR>::T;
    KnnParams p;
    fill_params(c, p, h_out, nbr, k_stride, use_guess);
    if (redo) {
        p.leaf_list = c->d_knn_redo;
        p.list_len = &c->d_cnt->knn_redo[0];
        p.work = &c->d_cnt->knn_redo[1];
    }
    auto kern = k_knn<R, NBR, TMA, G, CH, BATCH>;
    const size_t per_warp = knn_warp_bytes_t<R, K, G, BATCH>(p.kcap);
    int warps = 0, grid = 0;
    if (int rc = pick_shape(c, (const void*)kern, per_warp, &warps, &grid)) return rc;
    if (!redo) c->knn_grid = grid;
    cudaError_t e;
    if (!redo) {
        e = cudaMemsetAsync(&c->d_cnt->work[0], 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) return cuda_check(c, e, "knn work reset");
    }
    const int tidx = timer_begin(c, 1, s);
    kern<<<grid, warps * 32, (size_t)warps * per_warp, s>>>(p);
    timer_end(c, tidx, s);
    c->launches++;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(c, e, "knn launch");
    return SIDM_OK;
}

// the plain-load kernel-size search with the configured lane groups, chains
// and candidate loop (per staged leaf, or compacted batches)
template <class R>
int launch_tuned(sidm_ctx* c, void* h_out, bool use_guess, cudaStream_t s, bool redo = false)
{
    const int g = c->cfg.knn_groups > 0 ? c->cfg.knn_groups : kGroupsDefault;
    const int ch = c->cfg.knn_chains > 0 ? c->cfg.knn_chains : kChainsDefault;
    const bool batch = (c->cfg.knn_batch > 0 ? c->cfg.knn_batch : kBatchDefault) >= 2;
#define SIDM_KNN_CASE(GG, CC, BB) \
    if (g == GG && ch == CC && batch == BB) return launch_t<R, false, false, GG, CC, BB>(c, h_out, nullptr, 0, use_guess, s, redo);
    SIDM_KNN_CASE(2, 4, false) SIDM_KNN_CASE(4, 4, false) SIDM_KNN_CASE(8, 4, false) SIDM_KNN_CASE(4, 8, false)
    SIDM_KNN_CASE(2, 4, true) SIDM_KNN_CASE(4, 4, true) SIDM_KNN_CASE(8, 4, true) SIDM_KNN_CASE(4, 8, true)
#undef SIDM_KNN_CASE
    return set_err(c, SIDM_EINVAL, "knn_chains 8 takes knn_groups 4");
}

// warm-started search with the fixed-bound kernel, then the per-lane search
// (itself warm-started: a lane whose guess fails there is redone cold) of the
// leaves it could not finish or left to it
template <class R, int G>
int launch_warm(sidm_ctx* c, void* h_out, cudaStream_t s)
{
    using K = typename KeyOf<R, false>::T;
    KnnParams p;
    fill_params(c, p, h_out, nullptr, 0, true);
    auto kern = k_knn_warm<R, G>;
    const size_t per_warp = warm_warp_bytes<R, K, G>(p.kcap);
    int warps = 0, grid = 0;
    if (int rc = pick_shape(c, (const void*)kern, per_warp, &warps, &grid, kWarmMaxWarps)) return rc;
    c->knn_grid = grid;
    cudaError_t e = cudaMemsetAsync(&c->d_cnt->work[0], 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&c->d_cnt->knn_redo[0], 0, 2 * sizeof(unsigned int), s);
    if (e != cudaSuccess) return cuda_check(c, e, "knn work reset");
    const int tidx = timer_begin(c, 1, s);
    kern<<<grid, warps * 32, (size_t)warps * per_warp, s>>>(p, c->d_knn_redo, &c->d_cnt->knn_redo[0]);
    timer_end(c, tidx, s);
    c->launches++;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(c, e, "knn launch");
    return launch_tuned<R>(c, h_out, true, s, true);
}

template <class R>
int launch_warm_tuned(sidm_ctx* c, void* h_out, cudaStream_t s)
{
    const int g = c->cfg.knn_groups > 0 ? c->cfg.knn_groups : kGroupsDefault;
    return g == 2 ? launch_warm<R, 2>(c, h_out, s) : launch_warm<R, 4>(c, h_out, s);
}

}  // namespace

int launch_knn(sidm_ctx* c, void* h_out, uint32_t* nbr, int k_stride, bool use_guess, cudaStream_t s)
{
    if (c->lay.L == 0) return SIDM_OK;
    const bool tma = c->cfg.use_tma != 0;
    constexpr int G = kGroupsDefault, CH = kChainsDefault;   // neighbour lists and bulk copies: defaults
    // warm-started searches take the fixed-bound kernel unless the knobs ask for
    // bulk copies or the earlier combined kernel (knn_batch 1 or 2)
    const bool warm = use_guess && !tma && (c->cfg.knn_batch > 0 ? c->cfg.knn_batch : kBatchDefault) == 3;
    if (c->cfg.precision == SIDM_FP64) {
        if (nbr) return set_err(c, SIDM_EINVAL, "neighbour lists: mixed form only");
        if (warm) return launch_warm_tuned<double>(c, h_out, s);
        return tma ? launch_t<double, false, true, G, CH>(c, h_out, nullptr, 0, use_guess, s)
                   : launch_tuned<double>(c, h_out, use_guess, s);
    }
    if (nbr) return tma ? launch_t<float, true, true, G, CH>(c, nullptr, nbr, k_stride, false, s)
                        : launch_t<float, true, false, G, CH>(c, nullptr, nbr, k_stride, false, s);
    if (warm) return launch_warm_tuned<float>(c, h_out, s);
    return tma ? launch_t<float, false, true, G, CH>(c, h_out, nullptr, 0, use_guess, s)
               : launch_tuned<float>(c, h_out, use_guess, s);
}

}  // namespace sidm
