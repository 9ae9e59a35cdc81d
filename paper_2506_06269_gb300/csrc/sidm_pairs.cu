// sidm_pairs.cu -- (a2, a3) pair interaction probabilities and scatter draws.
//
// For every unordered pair of a halo with d_ij < h_i + h_j (Sect. 3.5: the
// geometric factor Lambda of the interaction probability is the overlap of
// the two spline kernels):
//   P_ij = (sigma(v_ij)/m) m_j v_ij Lambda_ij dt,  v_ij = |v_i - v_j|,
//   sigma/m = s0 or s0 / (1 + (v/w)^2)^2 (Sect. 3.8, Eq. vel_dep),
// and a counter-based Philox4x32-10 draw keyed by (seed; step, min id,
// max id, halo), so the draw is independent of thread order.  Event iff
// u = x0 2^-32 < P (no clamp: P >= 1 always fires).
//
// One warp per query leaf A; the tree walk visits leaves B >= A whose boxes
// are within h_max(A) + h_max(B), so each unordered pair is tested once, in
// the frame of the lower leaf.  The in-range test runs on a 32 x 32 block;
// in-range pairs are compacted into a per-warp queue of (slot i, slot j, d^2)
// that persists across candidate leaves, so the expensive part (sigma,
// Philox, Lambda) runs on full warps.  The Lambda table is read only for the
// pairs whose draw falls below an upper bound of P (see k_pairs).
#include "sidm_internal.cuh"
#include "sidm_tile.cuh"

namespace sidm {
namespace {

struct PairParams {
    int H, L;
    const int32_t* leaf_halo;
    const int32_t* leaf_off;
    const int64_t* halo_off;
    const int32_t* lvl_off;
    const int32_t* top;
    const HaloFrame* frame;
    const float4* cell;
    const float4* nlo;
    const float4* nhi;
    const void* P4;
    const void* V4;
    const void* lam;
    const sidm_xs* xs;
    const double* dt;
    const double* mass;
    uint32_t seed_lo, seed_hi, step_lo;
    uint32_t rk[20];    // Philox round keys of the seed
    const int32_t* bins;  // individual power-of-two steps (NULL: one step dt[h] for all)
    int n_bins, substep;
    double dt_max;
    sidm_event* ev;
    unsigned long long ev_cap;
    float* sump;
    int use_sump;
    double* dacc;       // local diagnostics: [5][nacc] kernel-weighted moments
    int64_t nacc;
    DevCounters* cnt;
    sidm_step_stats* st;
    double* evg;        // forward-dominated halos: G = m_j Lambda dt of each record (NULL: none allowed)
    double glx[8], glw[8];  // 8-point Gauss-Legendre rule on [-1, 1] (Lambda by quadrature)
};

// what one traversal of the in-range pairs computes
constexpr int kModeDraw = 0;        // draws, Lambda only below the bound of P
constexpr int kModeDrawExact = 1;   // draws, every P formed (per-particle sums of P)
constexpr int kModeDiag = 2;        // no draws: kernel-weighted moments for the local diagnostics

// spline kernel of Sect. 2, support h, normalised to one
template <class R>
__device__ __forceinline__ R spline_w(R d, R h)
{
    const R q = d / h;
    if (!(q < R(1))) return R(0);
    const R norm = R(8.0 / 3.14159265358979323846) / (h * h * h);
    if (q < R(0.5)) return norm * (R(1) - R(6) * q * q * (R(1) - q));
    const R t = R(1) - q;
    return norm * R(2) * t * t * t;
}

// pairs a lane queues per round, at most (a launch knob; swept on the GB300:
// 1, 2, 3, 4 -> 3.76, 3.64, 3.49, 3.47 ms), and the queue entries per warp, a
// power of two: a round adds up to 32 kPerRoundMax pairs to fewer than 32 waiting
constexpr int kPerRoundMax = 4;
constexpr int kQueue = 32 * (kPerRoundMax + 1) <= 64 ? 64 : 32 * (kPerRoundMax + 1) <= 128 ? 128 : 256;
static_assert(kQueue >= 32 * (kPerRoundMax + 1), "one round must fit behind the entries still waiting");

template <class R>
__device__ __forceinline__ uint32_t id_of(R w)
{
    if constexpr (sizeof(R) == 4) return __float_as_uint((float)w);
    else return (uint32_t)(double)w;
}

// individual power-of-two steps: a particle of bin b (step dt_max / 2^b) opens a
// step at sub-step s of the 2^(n_bins-1) sub-steps of the smallest bin iff s is
// a multiple of 2^(n_bins-1-b)
__device__ __forceinline__ bool step_opens(int b, int n_bins, int s)
{
    return (s & ((1 << (n_bins - 1 - b)) - 1)) == 0;
}

template <class R>
__device__ __forceinline__ float to_float_ru_p(R v)
{
    if constexpr (sizeof(R) == 8) return __double2float_ru((double)v);
    else return (float)v;
}

// per warp: staging buffers (the bulk-copy path lands a candidate leaf in the
// first; the plain path keeps the query leaf's own points there), the shifted
// candidate leaf, queue of in-range pairs (slot i, slot j), traversal stack,
// boxes of the nodes under test (32 lo + 32 hi)
template <class R, bool TMA>
constexpr size_t pair_warp_bytes()
{
    return (TileStageT<R, TMA>::bytes() + kQueue * 8 + kStack * 4 + 64 * 16 + 8 * 8 + 15) / 16 * 16;
}

// MODE kModeDrawExact: form P (and so Lambda) for every in-range pair
// (per-particle sums of P requested).  kModeDiag: no draws; each pair adds
// m W(d, h_i) and its velocity moments of j to particle i when d < h_i, and
// the same for j (the SPH sums of the local diagnostics).  kModeDraw: Lambda
// is looked up only when the draw lies below
// an upper bound of P: P_up uses kLamFUp in place of the interpolated table
// value, and since FP32/FP64 products round monotonically P <= P_up for the P
// that would have been formed, so a draw u >= P_up + 2e-6 decides "no event"
// and "not within 1e-6 of P" exactly as the full evaluation would.
template <class R, bool TMA, int MODE, int PR, bool DRAG>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2) k_pairs(PairParams p)
{
    static_assert(PR >= 1 && PR <= kPerRoundMax, "pairs per round");
    using V = typename Vec4<R>::T;
    using Stage = TileStageT<R, TMA>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char* base = smem + wid * pair_warp_bytes<R, TMA>();
    Stage st_pos(base);
    uint32_t* q_si = (uint32_t*)(base + Stage::bytes());
    uint32_t* q_sj = q_si + kQueue;
    int* stack = (int*)(q_sj + kQueue);
    float4* blo = (float4*)(stack + kStack);
    float4* bhi = blo + 32;
    // the warp's statistics (64-bit, added to once per query leaf, so the
    // per-lane counters of a leaf stay 32-bit registers): pairs, P > 1,
    // |P - u| < 1e-6, tests, Lambda lookups, tiles, most tiles of one leaf
    unsigned long long* wst = (unsigned long long*)(bhi + 32);
    if (lane < 8) wst[lane] = 0ull;
    st_pos.init(lane);
    const R* __restrict__ T = (const R*)p.lam;
    const V* __restrict__ P4 = (const V*)p.P4;
    const V* __restrict__ V4 = (const V*)p.V4;
    const uint32_t lt = (1u << lane) - 1u;


    while (true) {
        int leaf = 0;
        if (lane == 0) leaf = (int)atomicAdd(&p.cnt->work[1], 1u);
        leaf = __shfl_sync(0xffffffffu, leaf, 0);
        if (leaf >= p.L) break;
        const int h = p.leaf_halo[leaf];
        const int leaf0 = p.leaf_off[h];
        const int64_t hb = p.halo_off[h];
        const int64_t nh = p.halo_off[h + 1] - hb;
        const int64_t slot2u = hb - (int64_t)leaf0 * kLeaf;   // padded slot -> particle index
        const int A = leaf - leaf0;
        const int countA = (int)min((int64_t)kLeaf, nh - (int64_t)A * kLeaf);
        // with individual steps only particles whose step opens at this sub-step
        // take part; a leaf without such a particle has no pair to test
        const bool active = lane < countA &&
                            (!p.bins || step_opens(p.bins[hb + (int64_t)A * kLeaf + lane], p.n_bins, p.substep));
        if (p.bins && !__any_sync(0xffffffffu, active)) continue;
        const HaloFrame fr = p.frame[h];
        const float4 cA = p.cell[leaf];
        const sidm_xs xs = p.xs[h];
        const int kind = xs.kind;
        // forward-dominated halo: every in-range pair becomes a record (no draw);
        // only the instantiation for contexts with SIDM_FLAG_DRAG has room for them
        const bool drag = DRAG && MODE != kModeDiag && xs.angular != 0;
        if (!DRAG && MODE != kModeDiag && xs.angular != 0) {
            if (lane == 0) raise_status(p.cnt, SIDM_DEV_BAD_INPUT);
            continue;
        }
        const R pref = p.bins ? R(0) : (R)xs.s0 * (R)p.mass[h] * (R)p.dt[h];
        const R inv_w = kind == 1 ? R(1) / (R)xs.w : R(0);
        const float4 qlo = p.nlo[leaf], qhi = p.nhi[leaf];
        const float hmaxA = qlo.w;
        const uint32_t slotA = (uint32_t)leaf * kLeaf + lane;
        const V q = P4[slotA];
        // the queries in their own frame, for tiles tested candidate by lane (the
        // plain path stages tiles in registers, so the first staging buffer is free)
        V* qsh = st_pos.raw();
        if constexpr (!TMA) {
            __syncwarp();
            qsh[lane] = q;
            __syncwarp();
        }
        int qhead = 0, qn = 0;
        uint32_t n_pairs = 0u, n_gt1 = 0u, n_near = 0u, n_tested = 0u, n_lam = 0u, n_tiles = 0u;

        // d^2 of a queued pair, recomputed exactly as in the in-range test
        // (candidate shifted into the frame of the query's leaf)
        auto pair_d2 = [&](uint32_t si, uint32_t sj, const V& pi, const V& pj) -> R {
            R cx = pj.x, cy = pj.y, cz = pj.z;
            if constexpr (sizeof(R) == 4) {
                const float4 ci = p.cell[si / kLeaf], cj = p.cell[sj / kLeaf];
                cx = __fadd_rn(cx, __fsub_rn(cj.x, ci.x));
                cy = __fadd_rn(cy, __fsub_rn(cj.y, ci.y));
                cz = __fadd_rn(cz, __fsub_rn(cj.z, ci.z));
            }
            const R dx = sub_rn(cx, pi.x), dy = sub_rn(cy, pi.y), dz = sub_rn(cz, pi.z);
            return fma_rn(dz, dz, fma_rn(dy, dy, mul_rn(dx, dx)));
        };

        // P, draw and event (or the diagnostic moments) for queue entries
        // qhead .. qhead+nb-1, one per lane
        auto run_batch = [&](int nb) {
            __syncwarp();
            if constexpr (MODE == kModeDiag) {
                if (lane < nb) {
                    const int e = (qhead + lane) & (kQueue - 1);
                    const uint32_t si = q_si[e], sj = q_sj[e];
                    const V vi = V4[si], vj = V4[sj];
                    const V pi = P4[si], pj = P4[sj];
                    const R d2 = pair_d2(si, sj, pi, pj);
                    const R d = sqrt_rn(d2);
                    const R mh = (R)p.mass[h];
                    const int64_t ui = slot2u + si, uj = slot2u + sj;
                    if (d2 < mul_rn(pi.w, pi.w)) {
                        const double wt = (double)(mh * spline_w<R>(d, pi.w));
                        atomicAdd(p.dacc + ui, wt);
                        atomicAdd(p.dacc + p.nacc + ui, wt * (double)vj.x);
                        atomicAdd(p.dacc + 2 * p.nacc + ui, wt * (double)vj.y);
                        atomicAdd(p.dacc + 3 * p.nacc + ui, wt * (double)vj.z);
                        atomicAdd(p.dacc + 4 * p.nacc + ui,
                                  wt * ((double)vj.x * vj.x + (double)vj.y * vj.y + (double)vj.z * vj.z));
                    }
                    if (d2 < mul_rn(pj.w, pj.w)) {
                        const double wt = (double)(mh * spline_w<R>(d, pj.w));
                        atomicAdd(p.dacc + uj, wt);
                        atomicAdd(p.dacc + p.nacc + uj, wt * (double)vi.x);
                        atomicAdd(p.dacc + 2 * p.nacc + uj, wt * (double)vi.y);
                        atomicAdd(p.dacc + 3 * p.nacc + uj, wt * (double)vi.z);
                        atomicAdd(p.dacc + 4 * p.nacc + uj,
                                  wt * ((double)vi.x * vi.x + (double)vi.y * vi.y + (double)vi.z * vi.z));
                    }
                }
            } else if (lane < nb) {
                const int e = (qhead + lane) & (kQueue - 1);
                const uint32_t si = q_si[e], sj = q_sj[e];
                const V vi = V4[si], vj = V4[sj];
                const R hi = ((const R*)(P4 + si))[3], hj = ((const R*)(P4 + sj))[3];
                const R ux = vj.x - vi.x, uy = vj.y - vi.y, uz = vj.z - vi.z;
                const R v2 = ux * ux + uy * uy + uz * uz;
                const uint32_t ida = id_of<R>(vi.w), idb = id_of<R>(vj.w);
                const uint32_t a = min(ida, idb), b = max(ida, idb);
                const Philox4 x = philox4x32_10_rk(p.step_lo, a, b, (uint32_t)h, p.rk);
                // individual steps: the pair's longer step dt_max / 2^min(b_i, b_j)
                R prefp = pref;
                int bmin = 0;
                if (p.bins) {
                    bmin = min(p.bins[slot2u + si], p.bins[slot2u + sj]);
                    prefp = (R)xs.s0 * (R)p.mass[h] * (R)ldexp(p.dt_max, -bmin);
                }
                R P, pre, inv, u;
                bool need;
                if constexpr (sizeof(R) == 4) {
                    // P needs ~1e-6 relative accuracy only (the event decision below is
                    // exact for the P computed here): reciprocal square roots and
                    // approximate divisions are enough.
                    const float v = v2 > 0.f ? v2 * rsqrtf(v2) : 0.f;
                    float sig = 1.f;
                    if (kind == 1) { const float qq = v * inv_w; const float tt = 1.f + qq * qq; sig = __fdividef(1.f, tt * tt); }
                    pre = prefp * sig * v;
                    inv = __fdividef(1.f, fmaxf(hi, hj));
                    u = (R)((float)x.x[0] * 0x1p-32f);
                } else {
                    const R v = sqrt(v2);
                    R sig = R(1);
                    if (kind == 1) { const R qq = v * inv_w; const R tt = R(1) + qq * qq; sig = R(1) / (tt * tt); }
                    pre = prefp * sig * v;
                    inv = R(1) / (hi > hj ? hi : hj);
                    u = (R)ldexp((double)x.x[0], -32);
                }
                if constexpr (MODE == kModeDrawExact) {
                    need = true;
                } else {
                    const R P_up = pre * (R(kLamFUp) * inv * inv * inv);
                    need = drag || !(u >= P_up + R(2e-6));
                }
                P = R(0);
                R gfac = R(0);
                bool fire = false;
                if (need) {
                    ++n_lam;
                    const R d2 = pair_d2(si, sj, P4[si], P4[sj]);
                    R f;
                    if constexpr (sizeof(R) == 4) {
                        const float d = d2 > 0.f ? d2 * rsqrtf(d2) : 0.f;
                        f = lambda_f_fast(T, d, hi, hj, inv);
                    } else {
                        f = lambda_f<R>(T, sqrt_rn(d2), hi, hj);
                    }
                    P = pre * (f * inv * inv * inv);
                    if (drag) {
                        // the record keeps G = m_j Lambda dt; D = P / 3 at the step start.
                        // The turn's sine is the square root of a multiple of Lambda, so
                        // Lambda must be accurate relative to itself where it falls to
                        // zero, which neither the table nor an FP32 quadrature (its
                        // integrand cancels there) is: FP64 quadrature beyond half the
                        // support (everywhere in the FP64 form), the table inside, where
                        // Lambda > Lambda(0)/4 bounds its relative error
                        R lam = f * inv * inv * inv;
                        const R d2q = pair_d2(si, sj, P4[si], P4[sj]);
                        const R dq = sqrt_rn(d2q);
                        if (sizeof(R) == 8 || dq >= R(0.5) * (hi + hj))
                            lam = (R)lambda_quad<double>((double)dq, (double)hi, (double)hj, p.glx, p.glw);
                        fire = true;
                        P = pre * lam;
                        gfac = (R)p.mass[h] * lam * (p.bins ? (R)ldexp(p.dt_max, -bmin) : (R)p.dt[h]);
                        if (P > R(3)) ++n_gt1;
                    } else {
                        if constexpr (sizeof(R) == 4) fire = P >= R(1) || x.x[0] < (uint32_t)ceilf((float)P * 0x1p32f);
                        else fire = u < P;
                        if (P > R(1)) ++n_gt1;
                        if (fabs(P - u) < R(1e-6)) ++n_near;
                    }
                }
                const int64_t ui = slot2u + si, uj = slot2u + sj;
                if constexpr (MODE == kModeDrawExact) {
                    if (p.use_sump) {
                        // on individual steps a rate, scaled to dt_max (exact power of two)
                        const float ps = (float)(p.bins ? P * (R)ldexp(1.0, bmin) : P);
                        atomicAdd(p.sump + ui, ps);
                        atomicAdd(p.sump + uj, ps);
                    }
                }
                if (fire) {
                    const unsigned long long slot = atomicAdd(&p.cnt->ev_count, 1ull);
                    if (slot < p.ev_cap) {
                        sidm_event E;
                        E.key = ((unsigned long long)h << 54) | ((unsigned long long)a << 27) | (unsigned long long)b;
                        E.i = (uint32_t)(ida < idb ? ui : uj);
                        E.j = (uint32_t)(ida < idb ? uj : ui);
                        E.x1 = x.x[1];
                        E.x2 = x.x[2];
                        E.P = (float)P;
                        E.x0 = x.x[0];
                        p.ev[slot] = E;
                        if (drag) p.evg[slot] = (double)gfac;
                    }
                }
            }
            qhead = (qhead + nb) & (kQueue - 1);
            qn -= nb;
            __syncwarp();
        };

        // this lane's entry of candidate leaf Bl (the plain path loads it straight
        // into a register, so the walk can fetch the next leaf early)
        auto fetch = [&](int Bl) -> V {
            if constexpr (TMA) return V{};
            else return P4[(int64_t)(leaf0 + Bl) * kLeaf + lane];
        };
        // craw: fetch(Bl) (unused on the bulk-copy path, which stages the leaf here)
        auto process = [&](int Bl, bool mine, const V& craw) {
            const int Bg = leaf0 + Bl;
            ++n_tiles;
            const int countB = (int)min((int64_t)kLeaf, nh - (int64_t)Bl * kLeaf);
            V c;
            if constexpr (TMA) c = st_pos.load_lane(P4 + (int64_t)Bg * kLeaf, lane, p.cnt);
            else c = craw;
            if constexpr (sizeof(R) == 4) {
                const float4 cB = p.cell[Bg];
                c.x = __fadd_rn(c.x, __fsub_rn(cB.x, cA.x));
                c.y = __fadd_rn(c.y, __fsub_rn(cB.y, cA.y));
                c.z = __fadd_rn(c.z, __fsub_rn(cB.z, cA.z));
            }
            __syncwarp();
            V* tp = st_pos.shifted();
            tp[lane] = c;
            __syncwarp();
            const uint32_t slotB = (uint32_t)Bg * kLeaf;
            // candidates that cannot reach any query of A (box gap > h_t + hmax_A) are skipped
            float3 pc;
            if constexpr (sizeof(R) == 4) {
                pc = make_float3(__fadd_rn(cA.x, c.x), __fadd_rn(cA.y, c.y), __fadd_rn(cA.z, c.z));
            } else {
                pc = make_float3(__double2float_rn((double)c.x - fr.O[0]), __double2float_rn((double)c.y - fr.O[1]),
                                 __double2float_rn((double)c.z - fr.O[2]));
            }
            const float rc = __fadd_ru(__fmul_ru(__fadd_ru(to_float_ru_p<R>(c.w), hmaxA), 1.0f + 0x1p-20f), fr.margin);
            const uint32_t cmask = __ballot_sync(
                0xffffffffu, lane < countB && point_gap2_rd(pc, qlo, qhi) <= __fmul_ru(rc, rc) &&
                                 (!p.bins || step_opens(p.bins[hb + (int64_t)Bl * kLeaf + lane], p.n_bins, p.substep)));
            // (i) the pairs to test: queries that reach B (qmask) x candidates that
            //     can reach some query (cmask), inside A only candidate > query.  The
            //     warp loops over the smaller mask: lane = query, candidates from the
            //     staged tile (bits of okm = candidates), or lane = candidate, queries
            //     from their staged copy (bits = queries).  Same tests, same operands.
            const uint32_t qmask = __ballot_sync(0xffffffffu, mine);
            const bool by_cand = !TMA && __popc(qmask) < __popc(cmask);
            uint32_t okm = 0u, allow;
            if (!by_cand) {
                for (uint32_t mm = cmask; mm; mm &= mm - 1u) {
                    const int t = __ffs(mm) - 1;
                    const V pj = tp[t];
                    const R dx = sub_rn(pj.x, q.x), dy = sub_rn(pj.y, q.y), dz = sub_rn(pj.z, q.z);
                    const R d2 = fma_rn(dz, dz, fma_rn(dy, dy, mul_rn(dx, dx)));
                    const R hs = add_rn(q.w, pj.w);
                    okm |= (d2 < mul_rn(hs, hs) ? 1u : 0u) << t;
                }
                allow = mine ? cmask : 0u;
                if (Bl == A) allow &= 0xFFFFFFFEu << lane;
            } else {
                for (uint32_t mm = qmask; mm; mm &= mm - 1u) {
                    const int i = __ffs(mm) - 1;
                    const V qi = qsh[i];
                    const R dx = sub_rn(c.x, qi.x), dy = sub_rn(c.y, qi.y), dz = sub_rn(c.z, qi.z);
                    const R d2 = fma_rn(dz, dz, fma_rn(dy, dy, mul_rn(dx, dx)));
                    const R hs = add_rn(qi.w, c.w);
                    okm |= (d2 < mul_rn(hs, hs) ? 1u : 0u) << i;
                }
                allow = ((cmask >> lane) & 1u) ? qmask : 0u;
                if (Bl == A) allow &= (1u << lane) - 1u;
            }
            n_tested += (uint32_t)__popc(allow);
            okm &= allow;
            // queue entry of bit t: (query slot, candidate slot)
            const uint32_t own = by_cand ? slotB + lane : slotA;
            const uint32_t base = by_cand ? (uint32_t)leaf * kLeaf : slotB;
            // (ii) queue the pairs in rounds: every lane with pairs left adds up to
            //      PR, after the entries of the lanes below it
            for (uint32_t m = __ballot_sync(0xffffffffu, okm != 0u); m; m = __ballot_sync(0xffffffffu, okm != 0u)) {
                const int cnt = __popc(okm);
                int e = qhead + qn + __popc(m & lt);
                int c2 = __popc(m);
#pragma unroll
                for (int k = 2; k <= PR; ++k) {
                    const uint32_t mk = __ballot_sync(0xffffffffu, cnt >= k);
                    e += __popc(mk & lt);
                    c2 += __popc(mk);
                }
                const int take = min(cnt, PR);
                for (int k = 0; k < take; ++k, ++e) {
                    const int t = __ffs(okm) - 1;
                    okm &= okm - 1u;
                    q_si[e & (kQueue - 1)] = by_cand ? base + t : own;
                    q_sj[e & (kQueue - 1)] = by_cand ? own : base + t;
                }
                qn += c2;
                n_pairs += (uint32_t)c2;
                while (qn >= 32) run_batch(32);
            }
            __syncwarp();
        };

        // tree walk over leaves B >= A.  A node is visited iff some lane's point
        // lies within (h_i + hmax_node)(1 + 2^-20) + margin of the node's box.
        float3 pq;                                     // query point in the halo frame
        if constexpr (sizeof(R) == 4) {
            pq = make_float3(__fadd_rn(cA.x, (float)q.x), __fadd_rn(cA.y, (float)q.y), __fadd_rn(cA.z, (float)q.z));
        } else {
            pq = make_float3(__double2float_rn((double)q.x - fr.O[0]), __double2float_rn((double)q.y - fr.O[1]),
                             __double2float_rn((double)q.z - fr.O[2]));
        }
        const float hq = active ? to_float_ru_p<R>(q.w) : -INFINITY;
        // this lane's query reaches box c: within (h_i + hmax_node)(1 + 2^-20) + margin
        auto near_box = [&](int c) -> bool {
            const float4 lo = blo[c], hi = bhi[c];
            const float r = __fadd_ru(__fmul_ru(__fadd_ru(hq, lo.w), 1.0f + 0x1p-20f), fr.margin);
            return active && point_gap2_rd(pq, lo, hi) <= __fmul_ru(r, r);
        };
        // boxes of nodes g0 .. g0+n-1 (n <= kArity = 32), one per lane
        auto load_boxes = [&](int g0, int n) {
            __syncwarp();
            if (lane < n) { blo[lane] = p.nlo[g0 + lane]; bhi[lane] = p.nhi[g0 + lane]; }
            __syncwarp();
        };
        // bit c: some lane's query reaches box c (each lane keeps its own bits
        // for the leaves of this node).  Every query point lies in the leaf's
        // box, so a child farther from that box than the reach of the largest
        // h_i is out of reach of every lane: one box test per child (a lane
        // each) leaves the per-lane point tests to the children that pass it.
        float hqmax = hq;
        for (int o = 16; o > 0; o >>= 1) hqmax = fmaxf(hqmax, __shfl_xor_sync(0xffffffffu, hqmax, o));
        uint32_t lane_bits = 0u;
        auto accept = [&](int n, uint32_t eligible) -> uint32_t {
            bool reach = false;
            if (lane < n && ((eligible >> lane) & 1u)) {
                const float4 lo = blo[lane], hi = bhi[lane];
                const float r = __fadd_ru(__fmul_ru(__fadd_ru(hqmax, lo.w), 1.0f + 0x1p-20f), fr.margin);
                reach = box_gap2_rd(qlo, qhi, lo, hi) <= __fmul_ru(r, r);
            }
            const uint32_t near = __ballot_sync(0xffffffffu, reach);
            uint32_t bits = 0u;
            if (active)
                for (uint32_t m = near; m; m &= m - 1u) {
                    const int c = __ffs(m) - 1;
                    bits |= (near_box(c) ? 1u : 0u) << c;
                }
            lane_bits = bits;
            return __reduce_or_sync(0xffffffffu, bits);
        };
        // nodes whose subtree holds a leaf >= A (level lev, local indices first ..)
        auto eligible_mask = [&](int lev, int first, int n) -> uint32_t {
            return __ballot_sync(0xffffffffu, lane < n && ((int64_t)(first + lane + 1) << (kArityLog * lev)) > A);
        };
        // accepted leaves in index order; the next one is fetched before this one
        // is processed, so its load overlaps this leaf's tests
        auto visit_leaves = [&](uint32_t acc, int first) {
            if (acc == 0u) return;
            int c = __ffs(acc) - 1;
            acc &= acc - 1u;
            V cur = fetch(first + c);
            while (true) {
                const int cn = __ffs(acc) - 1;         // -1: none left
                acc &= acc - 1u;
                V nxt{};
                if (cn >= 0) nxt = fetch(first + cn);
                process(first + c, (lane_bits >> c) & 1u, cur);
                if (cn < 0) break;
                c = cn;
                cur = nxt;
            }
        };
        auto push = [&](uint32_t acc, int lev, int first, int& sp) -> bool {
            const int cnt = __popc(acc);
            if (sp + cnt > kStack) return false;
            // descending local index on the stack, so the lowest is visited first
            if ((acc >> lane) & 1u) stack[sp + cnt - 1 - __popc(acc & lt)] = (lev << 24) | (first + lane);
            sp += cnt;
            __syncwarp();
            return true;
        };
        const int top = p.top[h];
        const int Hp = p.H + 1;
        int sp = 0;
        bool failed = false;
        {
            const int nb = p.lvl_off[top * Hp + h];
            const int ntop = p.lvl_off[top * Hp + h + 1] - nb;
            load_boxes(nb, ntop);
            const uint32_t acc = accept(ntop, eligible_mask(top, 0, ntop));
            if (top == 0) visit_leaves(acc, 0);
            else if (!push(acc, top, 0, sp)) failed = true;
        }
        while (sp > 0 && !failed) {
            const int e = stack[--sp];
            __syncwarp();
            const int lev = e >> 24, idx = e & 0xFFFFFF;
            const int cl = lev - 1;
            const int cb = p.lvl_off[cl * Hp + h];
            const int cc = p.lvl_off[cl * Hp + h + 1] - cb;
            const int first = idx * kArity;
            const int nch = min(kArity, cc - first);
            load_boxes(cb + first, nch);
            const uint32_t acc = accept(nch, eligible_mask(cl, first, nch));
            if (cl == 0) visit_leaves(acc, first);
            else if (!push(acc, cl, first, sp)) failed = true;
        }
        // the queue outlives the staged tiles (entries are slots), so one partial
        // batch per query leaf remains
        if (qn > 0) run_batch(qn);
        if (failed && lane == 0) raise_status(p.cnt, SIDM_DEV_STACK);
        // this leaf's counts into the warp's 64-bit statistics (the per-lane
        // ones summed over the warp; pairs and tiles are the same in every lane)
        {
            const uint32_t g1 = __reduce_add_sync(0xffffffffu, n_gt1);
            const uint32_t nr = __reduce_add_sync(0xffffffffu, n_near);
            const uint32_t te = __reduce_add_sync(0xffffffffu, n_tested);
            const uint32_t la = __reduce_add_sync(0xffffffffu, n_lam);
            if (lane == 0) {
                wst[0] += n_pairs; wst[1] += g1; wst[2] += nr; wst[3] += te; wst[4] += la; wst[5] += n_tiles;
                wst[6] = max(wst[6], (unsigned long long)n_tiles);
            }
            __syncwarp();
        }
    }
    // warp totals -> step statistics
    if (lane == 0) {
        if (wst[0]) atomicAdd(&p.st->n_pairs, wst[0]);
        if (wst[1]) atomicAdd(&p.st->n_p_gt1, wst[1]);
        if (wst[2]) atomicAdd(&p.st->n_near, wst[2]);
        if (wst[3]) atomicAdd(&p.st->n_tested, wst[3]);
        atomicAdd(&p.cnt->diag[4], wst[5]);
        atomicMax(&p.cnt->diag[5], wst[6]);
        if (wst[4]) atomicAdd(&p.cnt->diag[6], wst[4]);
    }
    st_pos.finish(lane, p.cnt);
}

template <class R, bool TMA, int MODE, int PR = kPerRoundMax, bool DRAG = false>
int launch_t(sidm_ctx* c, uint64_t seed, uint64_t step, const sidm_xs* xs, const double* dt, const double* mass,
             sidm_step_stats* st, cudaStream_t s)
{
    PairParams p;
    const LayoutHost& L = c->lay;
    p.H = L.H; p.L = L.L;
    p.leaf_halo = c->d_leaf_halo; p.leaf_off = c->d_leaf_off; p.halo_off = c->d_halo_off;
    p.lvl_off = c->d_lvl_off; p.top = c->d_top; p.frame = c->d_frame; p.cell = c->d_cell;
    p.nlo = c->d_nlo; p.nhi = c->d_nhi; p.P4 = c->d_P4; p.V4 = c->d_V4; p.lam = c->d_lam;
    p.xs = xs; p.dt = dt; p.mass = mass;
    p.seed_lo = (uint32_t)seed; p.seed_hi = (uint32_t)(seed >> 32); p.step_lo = (uint32_t)step;
    for (int r = 0; r < 10; ++r) {
        p.rk[2 * r] = p.seed_lo + (uint32_t)r * 0x9E3779B9u;
        p.rk[2 * r + 1] = p.seed_hi + (uint32_t)r * 0xBB67AE85u;
    }
    p.ev = c->d_ev; p.ev_cap = (unsigned long long)c->cfg.event_cap;
    p.sump = c->d_sump; p.use_sump = (c->cfg.flags & SIDM_FLAG_SUM_P) ? 1 : 0;
    p.dacc = c->d_dacc; p.nacc = L.N;
    p.bins = c->step_bins; p.n_bins = c->step_nbins; p.substep = c->step_sub; p.dt_max = c->step_dtmax;
    p.cnt = c->d_cnt; p.st = st;
    p.evg = c->d_evg;
    for (int g = 0; g < 8; ++g) { p.glx[g] = c->gl8x[g]; p.glw[g] = c->gl8w[g]; }
    const int warps = c->pair_warps;
    const size_t smem = (size_t)warps * pair_warp_bytes<R, TMA>();
    auto kern = k_pairs<R, TMA, MODE, PR, DRAG>;
    int occ = 0;
    int rc = occupancy(c, (const void*)kern, warps * 32, smem, &occ);
    if (rc) return rc;
    cudaError_t e;
    if (occ < 1) return set_err(c, SIDM_ECAPACITY, "pair kernel does not fit on an SM");
    int grid = c->cfg.grid_ctas > 0 ? c->cfg.grid_ctas : c->sm_count * occ;
    grid = std::max(1, std::min(grid, (L.L + warps - 1) / warps));
    c->pair_grid = grid;
    e = cudaMemsetAsync(&c->d_cnt->work[1], 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return cuda_check(c, e, "pair work reset");
    const int tidx = MODE == kModeDiag ? -1 : timer_begin(c, 2, s);
    kern<<<grid, warps * 32, smem, s>>>(p);
    if (tidx >= 0) timer_end(c, tidx, s);
    c->launches++;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(c, e, "pair launch");
    return SIDM_OK;
}

}  // namespace

int launch_pairs(sidm_ctx* c, uint64_t seed, uint64_t step, const sidm_xs* xs, const double* dt, const double* mass,
                 sidm_step_stats* st, cudaStream_t s)
{
    if (c->lay.L == 0) return SIDM_OK;
    const bool tma = c->cfg.use_tma != 0;
    const bool exact = (c->cfg.flags & SIDM_FLAG_SUM_P) != 0;
    if (c->cfg.flags & SIDM_FLAG_DRAG) {                // forward-dominated halos allowed (plain loads)
        if (c->cfg.precision == SIDM_FP64)
            return exact ? launch_t<double, false, kModeDrawExact, kPerRoundMax, true>(c, seed, step, xs, dt, mass, st, s)
                         : launch_t<double, false, kModeDraw, kPerRoundMax, true>(c, seed, step, xs, dt, mass, st, s);
        return exact ? launch_t<float, false, kModeDrawExact, kPerRoundMax, true>(c, seed, step, xs, dt, mass, st, s)
                     : launch_t<float, false, kModeDraw, kPerRoundMax, true>(c, seed, step, xs, dt, mass, st, s);
    }
#define SIDM_PAIRS_DISPATCH(R)                                                                                   \
    if (exact) return tma ? launch_t<R, true, kModeDrawExact>(c, seed, step, xs, dt, mass, st, s)                \
                          : launch_t<R, false, kModeDrawExact>(c, seed, step, xs, dt, mass, st, s);              \
    if (tma) return launch_t<R, true, kModeDraw>(c, seed, step, xs, dt, mass, st, s);
    if (c->cfg.precision == SIDM_FP64) {
        SIDM_PAIRS_DISPATCH(double)
        return launch_t<double, false, kModeDraw>(c, seed, step, xs, dt, mass, st, s);
    }
    SIDM_PAIRS_DISPATCH(float)
#undef SIDM_PAIRS_DISPATCH
    // the hot path: pairs queued per lane and round as configured (a launch knob)
    switch (c->cfg.pair_per_round > 0 ? c->cfg.pair_per_round : kPerRoundMax) {
    case 1: return launch_t<float, false, kModeDraw, 1>(c, seed, step, xs, dt, mass, st, s);
    case 2: return launch_t<float, false, kModeDraw, 2>(c, seed, step, xs, dt, mass, st, s);
    case 3: return launch_t<float, false, kModeDraw, 3>(c, seed, step, xs, dt, mass, st, s);
    default: return launch_t<float, false, kModeDraw, 4>(c, seed, step, xs, dt, mass, st, s);
    }
}

int launch_pairs_diag(sidm_ctx* c, const sidm_xs* xs, const double* mass, cudaStream_t s)
{
    if (c->lay.L == 0) return SIDM_OK;
    if (c->cfg.precision == SIDM_FP64)
        return launch_t<double, false, kModeDiag>(c, 0, 0, xs, nullptr, mass, c->d_stats_own, s);
    return launch_t<float, false, kModeDiag>(c, 0, 0, xs, nullptr, mass, c->d_stats_own, s);
}

}  // namespace sidm
