// sidm_knn.cu -- (a1) kernel sizes: h_i = distance to the N_ngb-th nearest
// other particle of the halo (Sect. 2: "set by the next N_ngb neighbours";
// Eq. hDl: h is the radius of the sphere holding N_ngb particles).
//
// One warp per leaf of 32 consecutive Morton-ordered particles, one query per
// lane.  Candidate leaves are staged through shared memory (plain coalesced
// 128-bit loads, or bulk asynchronous copies with an mbarrier), shifted into
// the query leaf's frame, and every lane keeps a max-heap of its N_ngb
// smallest keys in shared memory.  The heap is first filled from the leaves
// next to the query leaf in Morton order, whose k-th distance bounds the
// search radius; the bounding-volume tree is then walked with that (shrinking)
// radius, skipping those leaves.  The result is the exact k-th smallest of the
// canonical distance, so it does not depend on tile order or launch shape.
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
    int work_slot;
};

template <class K> __device__ __forceinline__ K key_max();
template <> __device__ __forceinline__ uint32_t key_max<uint32_t>() { return 0xFFFFFFFFu; }
template <> __device__ __forceinline__ unsigned long long key_max<unsigned long long>() { return ~0ull; }

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

// replace the heap root (the largest of the k kept keys) by key and sift down
template <class K>
__device__ __forceinline__ void heap_replace(K* heap, int lane, int k, K key)
{
    int pos = 0;
    while (true) {
        int c = 2 * pos + 1;
        if (c >= k) break;
        K cv = heap[c * 32 + lane];
        if (c + 1 < k) {
            K c2 = heap[(c + 1) * 32 + lane];
            if (c2 > cv) { ++c; cv = c2; }
        }
        if (!(cv > key)) break;
        heap[pos * 32 + lane] = cv;
        pos = c;
    }
    heap[pos * 32 + lane] = key;
}

template <class K>
__device__ __forceinline__ void heap_sift(K* heap, int lane, int n)
{
    int pos = 0;
    const K key = heap[lane];
    while (true) {
        int c = 2 * pos + 1;
        if (c >= n) break;
        K cv = heap[c * 32 + lane];
        if (c + 1 < n) {
            K c2 = heap[(c + 1) * 32 + lane];
            if (c2 > cv) { ++c; cv = c2; }
        }
        if (!(cv > key)) break;
        heap[pos * 32 + lane] = cv;
        pos = c;
    }
    heap[pos * 32 + lane] = key;
}

template <class R>
__device__ __forceinline__ float to_float_ru(R v)
{
    if constexpr (sizeof(R) == 8) return __double2float_ru((double)v);
    else return (float)v;
}

template <class R, bool NBR, bool TMA>
__global__ void k_knn(KnnParams p)
{
    using V = typename Vec4<R>::T;
    using K = typename KeyOf<R, NBR>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t per_warp = knn_warp_bytes<R, K>(p.kcap);
    unsigned char* base = smem + wid * per_warp;
    TileStageT<R, TMA> stage(base);
    uint32_t* tids = (uint32_t*)(base + TileStageT<R, TMA>::bytes());
    int* stack = (int*)(tids + 32);
    K* heap = (K*)(stack + kStack);
    stage.init(lane);
    unsigned long long n_cand = 0ull, n_ins = 0ull, n_tiles_all = 0ull, n_tiles_max = 0ull;

    while (true) {
        int leaf = 0;
        if (lane == 0) leaf = (int)atomicAdd(&p.cnt->work[p.work_slot], 1u);
        leaf = __shfl_sync(0xffffffffu, leaf, 0);
        if (leaf >= p.L) break;
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
        const float4 cA = p.cell[leaf];
        const float4 qlo = p.nlo[leaf], qhi = p.nhi[leaf];
        const K kmax = key_max<K>();
        for (int t = 0; t < k; ++t) heap[t * 32 + lane] = kmax;
        K root = kmax;
        bool failed = false;
        unsigned long long n_tiles = 0ull;

        auto process = [&](int Bl, bool mine) {
            const int Bg = leaf0 + Bl;
            const int countB = (int)min((int64_t)kLeaf, nh - (int64_t)Bl * kLeaf);
            const V* tile = stage.load((const V*)p.P4 + (int64_t)Bg * kLeaf, lane, p.cnt);
            // shift the candidates into the query leaf's frame (exact shift)
            V c = tile[lane];
            if constexpr (sizeof(R) == 4) {
                const float4 cB = p.cell[Bg];
                c.x = __fadd_rn(c.x, __fsub_rn(cB.x, cA.x));
                c.y = __fadd_rn(c.y, __fsub_rn(cB.y, cA.y));
                c.z = __fadd_rn(c.z, __fsub_rn(cB.z, cA.z));
            }
            __syncwarp();
            V* sh = stage.shifted();
            sh[lane] = c;
            if (NBR) tids[lane] = p.ID[(int64_t)Bg * kLeaf + lane];
            __syncwarp();
            ++n_tiles;
            if (active && mine) {
                n_cand += (unsigned long long)countB;
                for (int t = 0; t < countB; ++t) {
                    if (Bl == A && t == lane) continue;
                    const V cj = sh[t];
                    const R dx = sub_rn(cj.x, q.x), dy = sub_rn(cj.y, q.y), dz = sub_rn(cj.z, q.z);
                    const R d2 = fma_rn(dz, dz, fma_rn(dy, dy, mul_rn(dx, dx)));
                    const K key = make_key<R, NBR>(d2, NBR ? tids[t] : 0u);
                    if (key < root) {
                        ++n_ins;
                        heap_replace<K>(heap, lane, k, key);
                        root = heap[lane];
                    }
                }
            }
            __syncwarp();
        };

        // 1) Morton-window leaves around A holding at least k+1 particles
        int wlo = A, whi = A;
        int64_t wcount = countA;
        while (wcount < k + 1 && (wlo > 0 || whi < nleaf - 1)) {
            if (whi < nleaf - 1) { ++whi; wcount += min((int64_t)kLeaf, nh - (int64_t)whi * kLeaf); }
            if (wcount < k + 1 && wlo > 0) { --wlo; wcount += kLeaf; }
        }
        for (int Bl = wlo; Bl <= whi; ++Bl) process(Bl, true);

        // 2) tree walk.  A node is visited iff the query point of some lane lies
        //    within that lane's current k-th distance (+ margin) of the node's box;
        //    accepted leaves are processed at once so the bound keeps shrinking.
        float3 pq;                                     // query point in the halo frame
        if constexpr (sizeof(R) == 4) {
            pq = make_float3(__fadd_rn(cA.x, (float)q.x), __fadd_rn(cA.y, (float)q.y), __fadd_rn(cA.z, (float)q.z));
        } else {
            pq = make_float3(__double2float_rn((double)q.x - fr.O[0]), __double2float_rn((double)q.y - fr.O[1]),
                             __double2float_rn((double)q.z - fr.O[2]));
        }
        auto my_r2 = [&]() -> float {
            if (!active) return -1.0f;
            float r = to_float_ru<R>(sqrt_ru(key_d2<R, NBR>(root)));
            r = __fadd_ru(__fmul_ru(r, 1.0f + 0x1p-20f), fr.margin);
            return __fmul_ru(r, r);
        };
        auto near = [&](int g, float r2) -> bool {
            return r2 >= 0.f && point_gap2_rd(pq, p.nlo[g], p.nhi[g]) <= r2;
        };
        auto visit_leaf = [&](int Bl) {
            const bool mine = near(leaf0 + Bl, my_r2());
            if (__any_sync(0xffffffffu, mine)) process(Bl, mine);
        };
        const int top = p.top[h];
        const int32_t* loff = p.lvl_off;
        const int Hp = p.H + 1;
        // Accepted nodes are visited nearest first (box gap to the query leaf),
        // so the k-th bound shrinks early.  rank = position among the accepted.
        auto order_rank = [&](uint32_t acc, int n, int g0) -> int {
            const bool mine_acc = lane < n && ((acc >> lane) & 1u);
            const float pr = mine_acc ? box_gap2_rd(qlo, qhi, p.nlo[g0 + lane], p.nhi[g0 + lane]) : INFINITY;
            int rank = 0;
            for (int j = 0; j < n; ++j) {
                const float pj = __shfl_sync(0xffffffffu, pr, j);
                if ((acc >> j) & 1u) rank += (pj < pr || (pj == pr && j < lane)) ? 1 : 0;
            }
            return rank;
        };
        auto visit_leaves_in_order = [&](uint32_t acc, int n, int first_local, int g0) {
            const int rank = order_rank(acc, n, g0);
            const int cnt = __popc(acc);
            for (int r = 0; r < cnt; ++r) {
                const uint32_t m = __ballot_sync(0xffffffffu, lane < n && ((acc >> lane) & 1u) && rank == r);
                visit_leaf(first_local + __ffs(m) - 1);
            }
        };
        auto push_in_order = [&](uint32_t acc, int n, int lev, int first_local, int g0, int& sp) -> bool {
            const int rank = order_rank(acc, n, g0);
            const int cnt = __popc(acc);
            if (sp + cnt > kStack) return false;
            if (lane < n && ((acc >> lane) & 1u)) stack[sp + cnt - 1 - rank] = (lev << 24) | (first_local + lane);
            sp += cnt;
            __syncwarp();
            return true;
        };
        int sp = 0;
        {
            const int nb = loff[top * Hp + h];
            const int ntop = loff[top * Hp + h + 1] - nb;
            const float r2 = my_r2();
            uint32_t acc = 0u;
            for (int c = 0; c < ntop; ++c) {
                if (top == 0 && c >= wlo && c <= whi) continue;
                if (__any_sync(0xffffffffu, near(nb + c, r2))) acc |= 1u << c;
            }
            if (top == 0) visit_leaves_in_order(acc, ntop, 0, nb);
            else if (!push_in_order(acc, ntop, top, 0, nb, sp)) failed = true;
        }
        while (sp > 0 && !failed) {
            const int e = stack[--sp];
            __syncwarp();
            const int lev = e >> 24, idx = e & 0xFFFFFF;
            const int cl = lev - 1;
            const int cb = loff[cl * Hp + h];
            const int cc = loff[cl * Hp + h + 1] - cb;
            const int first = idx * 8;
            const int nch = min(8, cc - first);
            const float r2 = my_r2();
            uint32_t acc = 0u;
            for (int c = 0; c < nch; ++c) {
                if (cl == 0 && first + c >= wlo && first + c <= whi) continue;
                if (__any_sync(0xffffffffu, near(cb + first + c, r2))) acc |= 1u << c;
            }
            if (cl == 0) visit_leaves_in_order(acc, nch, first, cb + first);
            else if (!push_in_order(acc, nch, cl, first, cb + first, sp)) failed = true;
        }
        if (failed && lane == 0) raise_status(p.cnt, SIDM_DEV_STACK);
        n_tiles_all += n_tiles;
        n_tiles_max = n_tiles > n_tiles_max ? n_tiles : n_tiles_max;

        // 3) outputs
        if (active) {
            const int64_t u = hb + (int64_t)A * kLeaf + lane;
            const R hval = sqrt_rn(key_d2<R, NBR>(root));
            if (p.h_out) {
                ((R*)p.h_out)[u] = hval;
                ((R*)((V*)p.P4 + (int64_t)leaf * kLeaf + lane))[3] = hval;
            }
            if constexpr (NBR) {
                for (int end = k - 1; end > 0; --end) {       // heap sort: ascending keys
                    const K t0 = heap[lane];
                    heap[lane] = heap[end * 32 + lane];
                    heap[end * 32 + lane] = t0;
                    heap_sift<K>(heap, lane, end);
                }
                for (int t = 0; t < k; ++t) p.nbr[u * p.k_stride + t] = (uint32_t)(heap[t * 32 + lane] & 0xFFFFFFFFull);
            }
        }
        __syncwarp();
    }
    // diagnostics: tiles, lane-level candidates, heap insertions, worst leaf
    for (int o = 16; o > 0; o >>= 1) {
        n_cand += __shfl_xor_sync(0xffffffffu, n_cand, o);
        n_ins += __shfl_xor_sync(0xffffffffu, n_ins, o);
    }
    if (lane == 0) {
        atomicAdd(&p.cnt->diag[0], n_tiles_all);
        atomicAdd(&p.cnt->diag[1], n_cand);
        atomicAdd(&p.cnt->diag[2], n_ins);
        atomicMax(&p.cnt->diag[3], n_tiles_max);
    }
    stage.finish(lane, p.cnt);
}

template <class R, bool NBR, bool TMA>
int launch_t(sidm_ctx* c, void* h_out, uint32_t* nbr, int k_stride, cudaStream_t s)
{
    using K = typename KeyOf<R, NBR>::T;
    KnnParams p;
    const LayoutHost& L = c->lay;
    p.H = L.H; p.L = L.L;
    p.leaf_halo = c->d_leaf_halo; p.leaf_off = c->d_leaf_off; p.halo_off = c->d_halo_off;
    p.lvl_off = c->d_lvl_off; p.top = c->d_top; p.ngb = c->d_ngb; p.frame = c->d_frame;
    p.cell = c->d_cell; p.nlo = c->d_nlo; p.nhi = c->d_nhi; p.P4 = c->d_P4; p.ID = c->d_ID;
    p.h_out = h_out; p.nbr = nbr; p.k_stride = k_stride; p.kcap = c->kmax_cur; p.cnt = c->d_cnt;
    p.work_slot = 0;
    const int warps = c->knn_warps;
    const size_t smem = (size_t)warps * knn_warp_bytes<R, K>(p.kcap);
    auto kern = k_knn<R, NBR, TMA>;
    int occ = 0;
    int rc = occupancy(c, (const void*)kern, warps * 32, smem, &occ);
    if (rc) return rc;
    cudaError_t e;
    if (occ < 1) return set_err(c, SIDM_ECAPACITY, "knn kernel does not fit on an SM (ngb_max too large for knn_warps)");
    int grid = c->cfg.grid_ctas > 0 ? c->cfg.grid_ctas : c->sm_count * occ;
    grid = std::max(1, std::min(grid, (L.L + warps - 1) / warps));
    c->knn_grid = grid;
    e = cudaMemsetAsync(&c->d_cnt->work[0], 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return cuda_check(c, e, "knn work reset");
    const int tidx = timer_begin(c, 1, s);
    kern<<<grid, warps * 32, smem, s>>>(p);
    timer_end(c, tidx, s);
    c->launches++;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(c, e, "knn launch");
    return SIDM_OK;
}

}  // namespace

int launch_knn(sidm_ctx* c, void* h_out, uint32_t* nbr, int k_stride, cudaStream_t s)
{
    if (c->lay.L == 0) return SIDM_OK;
    const bool tma = c->cfg.use_tma != 0;
    if (c->cfg.precision == SIDM_FP64) {
        if (nbr) return set_err(c, SIDM_EINVAL, "neighbour lists: mixed form only");
        return tma ? launch_t<double, false, true>(c, h_out, nullptr, 0, s)
                   : launch_t<double, false, false>(c, h_out, nullptr, 0, s);
    }
    if (nbr) return tma ? launch_t<float, true, true>(c, nullptr, nbr, k_stride, s)
                        : launch_t<float, true, false>(c, nullptr, nbr, k_stride, s);
    return tma ? launch_t<float, false, true>(c, h_out, nullptr, 0, s)
               : launch_t<float, false, false>(c, h_out, nullptr, 0, s);
}

}  // namespace sidm
