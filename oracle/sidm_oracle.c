/*
 * sidm_oracle.c -- plain, slow FP64 CPU oracle of the SIDM scattering pass.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * What it computes (Fischer, Yu & Dolag 2025, "Accurately simulating
 * core-collapse self-interacting dark matter halos"):
 *   Sect. 2   : spline kernel (Monaghan 1985), kernel size set adaptively by
 *               the next N_ngb neighbours, explicit energy and linear-momentum
 *               conservation of each scattering.
 *   Sect. 3.5 : geometric factor Lambda for the interaction probability (the
 *               kernel overlap); Eq. hDl ties h to the sphere holding N_ngb
 *               particles.
 *   Sect. 3.8 : velocity-dependent cross-section, Eq. vel_dep.
 *   Sect. 5   : the pairwise scheme conserves energy whatever the kernel,
 *               since every scatter conserves it on its own.
 *   App. A    : viscosity cross-section normalised to the total one for
 *               isotropic scattering (so sigma_V = sigma here).
 *   Sect. 3.5, Sect. 3.6, App. C : local diagnostics -- SPH density and
 *               velocity dispersion over the particle's kernel, the effective
 *               cross-section (Eq. effective_cross_section), h/l (Eq. hDl) and
 *               the Knudsen number (Eq. knudsen_number).
 * Readings where the paper is silent:
 *   h_i      = distance to the N_ngb-th nearest *other* particle of the halo,
 *              ties broken by id; the kernel support radius is h_i.
 *   W(r,h)   = 8/(pi h^3) {1-6q^2+6q^3 (q<1/2); 2(1-q)^3 (q<1); 0}, q=r/h.
 *   Lambda   = int W(|x-x_i|,h_i) W(|x-x_j|,h_j) d^3x  (symmetric overlap).
 *   P_ij     = (sigma(v_ij)/m) m_j v_ij Lambda_ij dt, v_ij=|v_i-v_j|; a pair
 *              is in range iff d_ij < h_i + h_j; each unordered pair once.
 *   draw     = Philox4x32-10 (Salmon et al., SC'11), key = seed, counter =
 *              (step mod 2^32, min id, max id, halo); u_k = x_k 2^-32;
 *              event iff u_0 < P (no clamp for P > 1).
 *   scatter  = isotropic in the pair's centre-of-mass frame:
 *              cos(theta) = 2 u_1 - 1, phi = 2 pi u_2; the particle with the
 *              smaller id gets v_cm + (m_j/M)|dv| n, the other v_cm - (m_i/M)|dv| n.
 *   multi-hit: events are accepted from step-start velocities and applied
 *              one after another in ascending (halo, min id, max id) order,
 *              each with the *current* velocities.
 *   forward-dominated (frictional) scattering, Sect. 3.8 with App. A: the
 *              limit theta -> 0 at fixed momentum transfer.  Every in-range
 *              pair interacts every step (no draw): its relative velocity
 *              u = v_i - v_j (i the smaller id) turns by the angle alpha with
 *              cos(alpha) = 1 - D, sin(alpha) = sqrt(D (2 - D)) (alpha = pi
 *              for D >= 2), D = (sigma_T/m) m_j |u| Lambda_ij dt, where
 *              sigma_T = sigma_V / 3 is the momentum-transfer cross-section of
 *              that limit at the given viscosity cross-section sigma_V
 *              (App. A: sigma_V = (3/2) int sin^2 dsigma, sigma_T =
 *              int (1 - cos) dsigma, both (1/2) int theta^2 dsigma at small
 *              angles), towards the projection onto u's normal plane of the
 *              isotropic Philox direction w (cos(theta) = 2 u_1 - 1,
 *              phi = 2 pi u_2), whose azimuth about u is uniform; |u| and
 *              v_cm are kept (energy and momentum conserved).  The mean
 *              change of u is the drag -D u; pairs are applied in ascending
 *              key order from the current velocities, with Lambda_ij, m_j and
 *              dt of the step start.
 *   mixed form: the FP32 pair distance is computed from FP32 offsets to
 *              power-of-two cell origins (see "canonical FP32 geometry").
 *
 * Parity pins (tests/test_oracle_*.py): brute-force kNN, Lambda normalised to
 * one, Lambda symmetry / support / small-kernel limit / Monte Carlo, Philox
 * known-answer vectors, per-event conservation, isotropy, the closed-form
 * collision rate of a uniform Maxwellian box, exact sums.
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off -fopenmp  (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LEAF 32           /* particles per leaf of the canonical geometry */
#define ORC_MBITS 17          /* Morton bits per axis                          */
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, from its published definition (Salmon et al. 2011):        */
/* round: (hi0,lo0)=M0*c0, (hi1,lo1)=M1*c2;                                   */
/*        c' = (hi1^c1^k0, lo1, hi0^c3^k1, lo0); key bumped by the Weyl pair  */
/*        between rounds.                                                     */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* Cubic spline kernel with compact support h, normalised to one (Sect. 2).  */
/* ------------------------------------------------------------------------- */
double orc_kernel_w(double r, double h)
{
    double q = r / h;
    if (q >= 1.0 || q < 0.0) return 0.0;
    double norm = 8.0 / (ORC_PI * h * h * h);
    if (q < 0.5) return norm * (1.0 - 6.0 * q * q + 6.0 * q * q * q);
    double t = 1.0 - q;
    return norm * 2.0 * t * t * t;
}

/* 8-point Gauss-Legendre nodes/weights on [-1,1] (exact to degree 15). */
static const double GL8_X[8] = {
    -0.9602898564975363, -0.7966664774136267, -0.5255324099163290, -0.1834346424956498,
     0.1834346424956498,  0.5255324099163290,  0.7966664774136267,  0.9602898564975363};
static const double GL8_W[8] = {
     0.1012285362903763,  0.2223810344533745,  0.3137066458778873,  0.3626837833783620,
     0.3626837833783620,  0.3137066458778873,  0.2223810344533745,  0.1012285362903763};

/* int_a^b s W(s,h) ds, piecewise GL (breakpoint h/2), exact for the spline. */
static double inner_sw(double a, double b, double h)
{
    if (b > h) b = h;
    if (a < 0.0) a = 0.0;
    if (b <= a) return 0.0;
    double brk[3] = {a, b, b};
    int nb = 2;
    if (0.5 * h > a && 0.5 * h < b) { brk[1] = 0.5 * h; brk[2] = b; nb = 3; }
    double acc = 0.0;
    for (int p = 0; p + 1 < nb; ++p) {
        double lo = brk[p], hi = brk[p + 1], m = 0.5 * (lo + hi), hw = 0.5 * (hi - lo);
        for (int g = 0; g < 8; ++g) {
            double s = m + hw * GL8_X[g];
            acc += GL8_W[g] * hw * s * orc_kernel_w(s, h);
        }
    }
    return acc;
}

static int cmp_dbl(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/*
 * Geometric factor Lambda(d; h_i, h_j) = int W_i W_j d^3x  (Sect. 3.5 reading),
 * in FP64.  Bipolar coordinates (r = |x-x_i|, s = |x-x_j|, d^3x = 2 pi r s
 * dr ds / d over |r-s| <= d <= r+s) give
 *   Lambda = (2 pi / d) int_0^{h_i} r W_i(r) [ int_{|r-d|}^{r+d} s W_j(s) ds ] dr.
 * The outer integrand is a polynomial between the breakpoints
 * {h_i/2, h_i, d, d +- h_j/2, d +- h_j, h_j/2 - d, h_j - d}; 8-point
 * Gauss-Legendre per piece is exact there (degree <= 9), as is the inner one.
 * For d -> 0 the limit 4 pi int r^2 W_i W_j dr is used.
 */
double orc_lambda(double d, double hi, double hj)
{
    if (d < 0.0) d = -d;
    if (d >= hi + hj) return 0.0;
    if (d < 1e-9 * (hi + hj)) {
        double top = hi < hj ? hi : hj;
        double brk[4] = {0.0, 0.5 * hi, 0.5 * hj, top};
        qsort(brk, 4, sizeof(double), cmp_dbl);
        double acc = 0.0;
        for (int p = 0; p < 3; ++p) {
            double lo = brk[p], up = brk[p + 1];
            if (up > top) up = top;
            if (up <= lo) continue;
            double m = 0.5 * (lo + up), hw = 0.5 * (up - lo);
            for (int g = 0; g < 8; ++g) {
                double r = m + hw * GL8_X[g];
                acc += GL8_W[g] * hw * r * r * orc_kernel_w(r, hi) * orc_kernel_w(r, hj);
            }
        }
        return 4.0 * ORC_PI * acc;
    }
    double lo = d - hj; if (lo < 0.0) lo = 0.0;
    double up = d + hj; if (up > hi) up = hi;
    if (up <= lo) return 0.0;
    double cand[11] = {lo, up, 0.5 * hi, hi, d, d - 0.5 * hj, d + 0.5 * hj,
                       d - hj, d + hj, 0.5 * hj - d, hj - d};
    double brk[11];
    int nb = 0;
    for (int c = 0; c < 11; ++c)
        if (cand[c] >= lo && cand[c] <= up) brk[nb++] = cand[c];
    qsort(brk, nb, sizeof(double), cmp_dbl);
    double acc = 0.0;
    for (int p = 0; p + 1 < nb; ++p) {
        double a = brk[p], b = brk[p + 1];
        if (b <= a) continue;
        double m = 0.5 * (a + b), hw = 0.5 * (b - a);
        for (int g = 0; g < 8; ++g) {
            double r = m + hw * GL8_X[g];
            double sl = fabs(r - d), su = r + d;
            acc += GL8_W[g] * hw * r * orc_kernel_w(r, hi) * inner_sw(sl, su, hj);
        }
    }
    return 2.0 * ORC_PI * acc / d;
}

/* Velocity-dependent cross-section per unit mass, Eq. vel_dep (Sect. 3.8);
 * kind 0: constant s0; kind 1: s0 / (1 + (v/w)^2)^2 with v the pair speed. */
double orc_sigma(int kind, double s0, double w, double v)
{
    if (kind == 0) return s0;
    double q = v / w;
    double t = 1.0 + q * q;
    return s0 / (t * t);
}

/* ------------------------------------------------------------------------- */
/* Canonical FP32 geometry of the mixed form.                                 */
/* Per halo: cube exponent E (2^E > largest bbox extent), origin O (per axis  */
/* a multiple of 2^E below the minimum), cube [O, O + 2^(E+1))^3.  Morton key */
/* of 3 x 17 bits, stable sort, leaves of 32 consecutive particles.  A leaf's */
/* frame origin is the corner c (relative to O) of the finest Morton cell     */
/* (edge 2^(E+1-17)) of its first particle, exact in FP32.                    */
/* Offsets o = RN32(RN64(x - (O + c))).                                       */
/* Distance from query i (leaf A) to j (leaf B):                              */
/*   s = c_B - c_A (exact), dx = RN32(RN32(o_j + s) - o_i),                   */
/*   d2 = fmaf(dz,dz, fmaf(dy,dy, dx*dx)).                                    */
/* A pair uses the frame of its lower leaf (Morton order).                    */
/* ------------------------------------------------------------------------- */
typedef struct {
    int n;                 /* particles in the halo                          */
    int nleaf;
    int E;
    double O[3];
    uint32_t* order;       /* sorted position -> local input index           */
    uint32_t* rank;        /* local input index -> sorted position           */
    float* off;            /* [3][n] offsets by local input index            */
    float* cell;           /* [3][nleaf] cell origins relative to O          */
} orc_geom;

static uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1FFFFFu, r = 0;
    for (int b = 0; b < 21; ++b) r |= ((x >> b) & 1u) << (3 * b);
    return r;
}

/* Stable LSD radix sort of 0..n-1 by a 64-bit key (13-bit digits over the
 * key's 51 Morton bits): order[s] = index of the s-th smallest key, equal keys
 * in input order. */
static void sort_by_key_stable(int n, const uint64_t* key, uint32_t* order)
{
    const int bits = 13, nb = 1 << 13;
    uint32_t* tmp = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    size_t* cnt = (size_t*)malloc(sizeof(size_t) * (size_t)nb);
    for (int i = 0; i < n; ++i) order[i] = (uint32_t)i;
    for (int shift = 0; shift < 3 * ORC_MBITS; shift += bits) {
        memset(cnt, 0, sizeof(size_t) * (size_t)nb);
        for (int s = 0; s < n; ++s) cnt[(key[order[s]] >> shift) & (uint64_t)(nb - 1)]++;
        size_t run = 0;
        for (int d = 0; d < nb; ++d) { size_t c = cnt[d]; cnt[d] = run; run += c; }
        for (int s = 0; s < n; ++s) tmp[cnt[(key[order[s]] >> shift) & (uint64_t)(nb - 1)]++] = order[s];
        memcpy(order, tmp, sizeof(uint32_t) * (size_t)n);
    }
    free(cnt);
    free(tmp);
}

static void geom_build(orc_geom* g, int n, const double* px, const double* py, const double* pz)
{
    const double* p[3] = {px, py, pz};
    memset(g, 0, sizeof(*g));
    g->n = n;
    g->nleaf = (n + ORC_LEAF - 1) / ORC_LEAF;
    double mn[3], mx[3], ext = 0.0;
    for (int a = 0; a < 3; ++a) {
        mn[a] = INFINITY; mx[a] = -INFINITY;
        for (int i = 0; i < n; ++i) { if (p[a][i] < mn[a]) mn[a] = p[a][i]; if (p[a][i] > mx[a]) mx[a] = p[a][i]; }
        if (n > 0 && mx[a] - mn[a] > ext) ext = mx[a] - mn[a];
    }
    int E = 0;
    if (ext > 0.0) frexp(ext, &E);            /* ext = m 2^E, m in [1/2,1) => 2^E > ext */
    g->E = E;
    for (int a = 0; a < 3; ++a) g->O[a] = n > 0 ? ldexp(floor(ldexp(mn[a], -E)), E) : 0.0;
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (n ? n : 1));
    uint32_t* q = (uint32_t*)malloc(sizeof(uint32_t) * 3 * (n ? n : 1));
    const uint32_t qmax = (1u << ORC_MBITS) - 1u;
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            double t = ldexp(p[a][i] - g->O[a], ORC_MBITS - E - 1);
            double f = floor(t);
            uint32_t v = f <= 0.0 ? 0u : (f >= (double)qmax ? qmax : (uint32_t)f);
            q[3 * i + a] = v;
        }
        key[i] = spread3(q[3 * i]) | (spread3(q[3 * i + 1]) << 1) | (spread3(q[3 * i + 2]) << 2);
    }
    g->order = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    g->rank = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    sort_by_key_stable(n, key, g->order);
    for (int s = 0; s < n; ++s) g->rank[g->order[s]] = (uint32_t)s;
    g->cell = (float*)malloc(sizeof(float) * 3 * (g->nleaf > 0 ? (size_t)g->nleaf : 1u));
    g->off = (float*)malloc(sizeof(float) * 3 * (n ? n : 1));
    const double fine = ldexp(1.0, E + 1 - ORC_MBITS);   /* finest Morton cell */
    for (int L = 0; L < g->nleaf; ++L) {
        int s0 = L * ORC_LEAF, s1 = s0 + ORC_LEAF - 1;
        if (s1 >= n) s1 = n - 1;
        uint32_t fi = g->order[s0];
        for (int a = 0; a < 3; ++a)
            g->cell[3 * L + a] = (float)((double)q[3 * fi + a] * fine);
        for (int s = s0; s <= s1; ++s) {
            uint32_t i = g->order[s];
            for (int a = 0; a < 3; ++a) {
                double C = g->O[a] + (double)g->cell[3 * L + a];
                g->off[3 * i + a] = (float)(p[a][i] - C);
            }
        }
    }
    free(key);
    free(q);
}

static void geom_free(orc_geom* g)
{
    free(g->order); free(g->rank); free(g->cell); free(g->off);
    memset(g, 0, sizeof(*g));
}

/* canonical FP32 squared distance from a point of offset oi in a leaf with
 * frame origin cA to a point of offset oj in a leaf with origin cB, in the
 * frame cA */
static float d2_mixed_core(const float* cA, const float* oi, const float* cB, const float* oj)
{
    volatile float dx[3];
    for (int a = 0; a < 3; ++a) {
        float s = cB[a] - cA[a];                                  /* exact */
        float t = oj[a] + s;
        dx[a] = t - oi[a];
    }
    float xx = dx[0] * dx[0];
    return fmaf(dx[2], dx[2], fmaf(dx[1], dx[1], xx));
}

/* canonical FP32 squared distance from i (its leaf frame) to j; local indices */
static float d2_mixed(const orc_geom* g, uint32_t i, uint32_t j)
{
    int A = (int)(g->rank[i] / ORC_LEAF), B = (int)(g->rank[j] / ORC_LEAF);
    return d2_mixed_core(g->cell + 3 * A, g->off + 3 * (size_t)i, g->cell + 3 * B, g->off + 3 * (size_t)j);
}

static double d2_fp64_core(const double* xi, const double* xj)
{
    double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
    double xx = dx * dx;
    return fma(dz, dz, fma(dy, dy, xx));
}

static double d2_fp64(const double* px, const double* py, const double* pz, uint32_t i, uint32_t j)
{
    const double xi[3] = {px[i], py[i], pz[i]}, xj[3] = {px[j], py[j], pz[j]};
    return d2_fp64_core(xi, xj);
}

/* float/double -> order-preserving unsigned bits (non-negative values) */
static uint32_t fbits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static uint64_t dbits(double f) { uint64_t u; memcpy(&u, &f, 8); return u; }

/* ------------------------------------------------------------------------- */
/* k-d tree over the particles of a halo: a plain search accelerator.  Every  */
/* search below returns what an exhaustive scan over all particles returns    */
/* (the tests pin both against brute force); the tree only skips boxes that   */
/* provably hold no candidate.  Nodes split their particles at the median of  */
/* the widest axis of their bounding box; leaves hold at most ORC_KD_LEAF.    */
/* ------------------------------------------------------------------------- */
#define ORC_KD_LEAF 16

typedef struct {
    double lo[3], hi[3];   /* bounding box of the node's particles (FP64)     */
    double hmax;           /* largest kernel size in the node (pair searches) */
    int start, count;      /* items[start .. start + count)                   */
    int left, right;       /* children, -1 at a leaf                          */
} orc_kdnode;

typedef struct {
    int n, nnode;
    orc_kdnode* node;
    int* items;            /* local particle indices                          */
    /* copies in item order, so that a leaf's candidates are read from       */
    /* consecutive memory (kd_attach; NULL until then)                        */
    float* toff;           /* [n][3] canonical offsets (mixed form)           */
    int* tleaf;            /* [n] canonical leaf (mixed form)                 */
    double* tpos;          /* [n][3] FP64 positions (FP64 form)               */
    uint32_t* tid;         /* [n] ids                                         */
} orc_kdtree;

/* reorder items[lo..hi) so that the element of rank m (by coordinate c) sits
 * at m, smaller ones before it and larger ones after it (quickselect) */
static void kd_select(int* it, int lo, int hi, int m, const double* c)
{
    while (hi - lo > 1) {
        const double piv = c[it[lo + (hi - lo) / 2]];
        int i = lo, j = hi - 1;
        while (i <= j) {
            while (c[it[i]] < piv) ++i;
            while (c[it[j]] > piv) --j;
            if (i <= j) { int t = it[i]; it[i] = it[j]; it[j] = t; ++i; --j; }
        }
        if (m <= j) hi = j + 1;
        else if (m >= i) lo = i;
        else return;
    }
}

static int kd_build_node(orc_kdtree* T, const double* const p[3], const double* h, int start, int count)
{
    int id;
    #pragma omp atomic capture
    id = T->nnode++;
    orc_kdnode* nd = &T->node[id];
    nd->start = start; nd->count = count; nd->left = nd->right = -1;
    nd->hmax = 0.0;
    for (int a = 0; a < 3; ++a) { nd->lo[a] = INFINITY; nd->hi[a] = -INFINITY; }
    for (int t = start; t < start + count; ++t) {
        const int i = T->items[t];
        for (int a = 0; a < 3; ++a) {
            if (p[a][i] < nd->lo[a]) nd->lo[a] = p[a][i];
            if (p[a][i] > nd->hi[a]) nd->hi[a] = p[a][i];
        }
        if (h && h[i] > nd->hmax) nd->hmax = h[i];
    }
    if (count <= ORC_KD_LEAF) return id;
    int ax = 0;
    for (int a = 1; a < 3; ++a) if (nd->hi[a] - nd->lo[a] > nd->hi[ax] - nd->lo[ax]) ax = a;
    const int half = count / 2;
    kd_select(T->items, start, start + count, start + half, p[ax]);
    int l, r;
    if (count > (1 << 16)) {               /* large subtrees are built in parallel */
        #pragma omp task shared(l)
        l = kd_build_node(T, p, h, start, half);
        r = kd_build_node(T, p, h, start + half, count - half);
        #pragma omp taskwait
    } else {
        l = kd_build_node(T, p, h, start, half);
        r = kd_build_node(T, p, h, start + half, count - half);
    }
    nd->left = l;                          /* T->node is sized up front, never moved */
    nd->right = r;
    return id;
}

/* h may be NULL (no per-node kernel sizes).  Node ids depend on the thread
 * schedule; the tree's shape and every search result do not. */
static void kd_build(orc_kdtree* T, int n, const double* px, const double* py, const double* pz, const double* h)
{
    const double* p[3] = {px, py, pz};
    memset(T, 0, sizeof(*T));
    T->n = n;
    T->items = (int*)malloc(sizeof(int) * (n ? n : 1));
    for (int i = 0; i < n; ++i) T->items[i] = i;
    /* leaves hold at least ORC_KD_LEAF / 2 particles (or all n <= ORC_KD_LEAF) */
    T->node = (orc_kdnode*)malloc(sizeof(orc_kdnode) * (size_t)(2 * (n / (ORC_KD_LEAF / 2) + 1)));
    if (n > 0) {
        #pragma omp parallel
        #pragma omp single
        kd_build_node(T, p, h, 0, n);
    }
}

static void kd_attach(orc_kdtree* T, const orc_geom* g, int mode, const double* px, const double* py,
                      const double* pz, const uint32_t* ids)
{
    const int n = T->n;
    T->tid = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    if (mode == 0) {
        T->toff = (float*)malloc(sizeof(float) * 3 * (size_t)(n ? n : 1));
        T->tleaf = (int*)malloc(sizeof(int) * (n ? n : 1));
    } else {
        T->tpos = (double*)malloc(sizeof(double) * 3 * (size_t)(n ? n : 1));
    }
    #pragma omp parallel for schedule(static)
    for (int t = 0; t < n; ++t) {
        const int j = T->items[t];
        T->tid[t] = ids[j];
        if (mode == 0) {
            T->tleaf[t] = (int)(g->rank[j] / ORC_LEAF);
            for (int a = 0; a < 3; ++a) T->toff[3 * (size_t)t + a] = g->off[3 * (size_t)j + a];
        } else {
            T->tpos[3 * (size_t)t] = px[j]; T->tpos[3 * (size_t)t + 1] = py[j]; T->tpos[3 * (size_t)t + 2] = pz[j];
        }
    }
}

static void kd_free(orc_kdtree* T)
{
    free(T->node); free(T->items); free(T->toff); free(T->tleaf); free(T->tpos); free(T->tid);
    memset(T, 0, sizeof(*T));
}

/* squared FP64 distance from x to the node's box (0 inside) */
static double kd_box_d2(const orc_kdnode* nd, const double x[3])
{
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        double g = 0.0;
        if (x[a] < nd->lo[a]) g = nd->lo[a] - x[a];
        else if (x[a] > nd->hi[a]) g = x[a] - nd->hi[a];
        s += g * g;
    }
    return s;
}

/* ------------------------------------------------------------------------- */
/* kNN kernel size h_i (Sect. 2: set by the next N_ngb neighbours).          */
/* Exact k-th smallest of the total order (d2, id) over other particles of   */
/* the halo.  mode 0: mixed (canonical FP32 d2), mode 1: FP64.               */
/* Outputs per local particle (input order): h (as double), d2k bits, and    */
/* optionally the k neighbour ids in ascending (d2, id) order.               */
/* brute != 0 scans all particles (O(N^2)); otherwise the k-d tree.         */
/* ------------------------------------------------------------------------- */
typedef struct { uint64_t d; uint32_t id; uint32_t idx; } knn_ent;

static int ent_less(const knn_ent* a, const knn_ent* b)
{
    if (a->d != b->d) return a->d < b->d;
    return a->id < b->id;
}

static void topk_insert(knn_ent* list, int* cnt, int k, knn_ent e)
{
    if (*cnt == k && !ent_less(&e, &list[k - 1])) return;
    int pos = *cnt < k ? (*cnt)++ : k - 1;
    while (pos > 0 && ent_less(&e, &list[pos - 1])) { list[pos] = list[pos - 1]; --pos; }
    list[pos] = e;
}

/* The k nearest other particles of particle i, sorted by (d^2, id), into
 * list[0..k); returns how many were found (k unless the halo is too small).
 * brute: every particle is a candidate.  Otherwise the k-d tree is walked,
 * nearer child first, and a box is skipped once the list holds k entries and
 * the box lies farther (exact FP64 distance) than the k-th entry's distance
 * with a margin of 1e-5 relative plus absmargin, which covers the difference
 * between the canonical FP32 distance and the exact one. */
static int knn_one(int i, int n, const double* px, const double* py, const double* pz, const uint32_t* ids,
                   int k, int mode, int brute, const orc_geom* g, const orc_kdtree* T, double absmargin,
                   knn_ent* list)
{
    int cnt = 0;
    if (brute) {
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            knn_ent e;
            e.d = mode == 0 ? (uint64_t)fbits(d2_mixed(g, (uint32_t)i, (uint32_t)j))
                            : dbits(d2_fp64(px, py, pz, (uint32_t)i, (uint32_t)j));
            e.id = ids[j]; e.idx = (uint32_t)j;
            topk_insert(list, &cnt, k, e);
        }
        return cnt;
    }
    const double xi[3] = {px[i], py[i], pz[i]};
    const float* cA = mode == 0 ? g->cell + 3 * (size_t)(g->rank[i] / ORC_LEAF) : NULL;
    const float* oi = mode == 0 ? g->off + 3 * (size_t)i : NULL;
    int stack[128], sp = 0;
    if (T->nnode > 0) stack[sp++] = 0;
    while (sp > 0) {
        const orc_kdnode* nd = &T->node[stack[--sp]];
        if (cnt == k) {
            double kth;
            if (mode == 0) { float f; uint32_t u = (uint32_t)list[k - 1].d; memcpy(&f, &u, 4); kth = sqrt((double)f); }
            else { double f; uint64_t u = list[k - 1].d; memcpy(&f, &u, 8); kth = sqrt(f); }
            const double lim = kth * (1.0 + 1e-5) + absmargin;
            if (kd_box_d2(nd, xi) > lim * lim) continue;
        }
        if (nd->left < 0) {
            for (int t = nd->start; t < nd->start + nd->count; ++t) {
                const int j = T->items[t];
                if (j == i) continue;
                knn_ent e;
                e.d = mode == 0 ? (uint64_t)fbits(d2_mixed_core(cA, oi, g->cell + 3 * (size_t)T->tleaf[t],
                                                                T->toff + 3 * (size_t)t))
                                : dbits(d2_fp64_core(xi, T->tpos + 3 * (size_t)t));
                e.id = T->tid[t]; e.idx = (uint32_t)j;
                topk_insert(list, &cnt, k, e);
            }
            continue;
        }
        const int l = nd->left, r = nd->right;
        const int near_l = kd_box_d2(&T->node[l], xi) <= kd_box_d2(&T->node[r], xi);
        stack[sp++] = near_l ? r : l;          /* the nearer child is popped first */
        stack[sp++] = near_l ? l : r;
    }
    return cnt;
}

int orc_knn_halo(int n, const double* px, const double* py, const double* pz, const uint32_t* ids,
                 int k, int mode, int brute, const uint8_t* query_mask,
                 double* h_out, uint64_t* d2k_bits_out, uint32_t* nbr_ids_out)
{
    if (k < 1 || k > n - 1) return -1;
    orc_geom g; memset(&g, 0, sizeof(g));
    if (mode == 0) geom_build(&g, n, px, py, pz);
    orc_kdtree T; memset(&T, 0, sizeof(T));
    if (!brute) {
        kd_build(&T, n, px, py, pz, NULL);
        kd_attach(&T, &g, mode, px, py, pz, ids);
    }
    int err = 0;
    /* the canonical FP32 distance is within (cube edge) * 2^-22 of the exact one */
    const double absmargin = mode == 0 ? ldexp(1.0, g.E + 1 - 20) : 0.0;
    #pragma omp parallel
    {
        knn_ent* list = (knn_ent*)malloc(sizeof(knn_ent) * (size_t)k);
        #pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            if (query_mask && !query_mask[i]) continue;
            int cnt = knn_one(i, n, px, py, pz, ids, k, mode, brute, &g, &T, absmargin, list);
            if (cnt < k) {
                #pragma omp atomic write
                err = -2;
                continue;
            }
            if (mode == 0) {
                float f; uint32_t u = (uint32_t)list[k - 1].d; memcpy(&f, &u, 4);
                h_out[i] = (double)sqrtf(f);
            } else {
                double f; uint64_t u = list[k - 1].d; memcpy(&f, &u, 8);
                h_out[i] = sqrt(f);
            }
            if (d2k_bits_out) d2k_bits_out[i] = list[k - 1].d;
            if (nbr_ids_out)
                for (int t = 0; t < k; ++t) nbr_ids_out[(size_t)i * k + t] = list[t].id;
        }
        free(list);
    }
    if (!brute) kd_free(&T);
    if (mode == 0) geom_free(&g);
    return err;
}

/* Kernel sizes of a list of particles for every N_ngb = 1..k at once: for the
 * t-th listed particle i = qidx[t], h_out[t*k + r] is the distance to its
 * (r+1)-th nearest other particle (same distance and order as orc_knn_halo),
 * from one geometry and tree build (test sampling of very large halos). */
int orc_knn_sample(int n, const double* px, const double* py, const double* pz, const uint32_t* ids,
                   int k, int mode, int64_t nq, const int64_t* qidx, double* h_out)
{
    if (k < 1 || k > n - 1) return -1;
    orc_geom g; memset(&g, 0, sizeof(g));
    if (mode == 0) geom_build(&g, n, px, py, pz);
    orc_kdtree T;
    kd_build(&T, n, px, py, pz, NULL);
    kd_attach(&T, &g, mode, px, py, pz, ids);
    int err = 0;
    const double absmargin = mode == 0 ? ldexp(1.0, g.E + 1 - 20) : 0.0;
    #pragma omp parallel
    {
        knn_ent* list = (knn_ent*)malloc(sizeof(knn_ent) * (size_t)k);
        #pragma omp for schedule(dynamic, 1)
        for (int64_t t = 0; t < nq; ++t) {
            const int i = (int)qidx[t];
            int cnt = knn_one(i, n, px, py, pz, ids, k, mode, 0, &g, &T, absmargin, list);
            if (cnt < k) {
                #pragma omp atomic write
                err = -2;
                continue;
            }
            for (int r = 0; r < k; ++r) {
                if (mode == 0) {
                    float f; uint32_t u = (uint32_t)list[r].d; memcpy(&f, &u, 4);
                    h_out[t * k + r] = (double)sqrtf(f);
                } else {
                    double f; uint64_t u = list[r].d; memcpy(&f, &u, 8);
                    h_out[t * k + r] = sqrt(f);
                }
            }
        }
        free(list);
    }
    kd_free(&T);
    if (mode == 0) geom_free(&g);
    return err;
}

/* ------------------------------------------------------------------------- */
/* Pair probabilities and draws (Sect. 3.5, Eq. vel_dep).                    */
/* Every unordered in-range pair of the halo once.  Mixed: range test         */
/* d2 < RN32(RN32(h_i+h_j)^2) on the canonical FP32 d2 in the lower leaf's   */
/* frame; FP64: d2 < (h_i+h_j)^2.  Each pair is evaluated in one orientation, */
/* (a, b) with h_a > h_b or (h_a == h_b and a < b); Lambda uses the FP64      */
/* distance of the FP64 positions.  The partners of a particle are found      */
/* with the k-d tree: a box is skipped if it lies farther (exact FP64) than   */
/* (h_i + largest h in the box)(1 + 1e-5) plus the canonical-distance margin. */
/* pair_mask (may be NULL): evaluate only the pairs with an endpoint i whose  */
/* pair_mask[i] is non-zero (test sampling at full size; the arithmetic of   */
/* every evaluated pair is unchanged).                                        */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint64_t key;     /* halo<<54 | min id<<27 | max id                       */
    uint32_t i, j;    /* local input indices; i has the smaller id            */
    uint32_t x1, x2;  /* Philox words for the scattering direction           */
    double P, u;
} orc_event;

typedef struct {
    int64_t n_pairs, n_events, n_p_gt1, n_near;
    double max_sum_p;
} orc_pair_stats;

/* Individual power-of-two time steps: a particle in bin b (step dt_max / 2^b)
 * opens a step at sub-step s (of 2^(n_bins-1) sub-steps of the smallest bin)
 * iff s is a multiple of 2^(n_bins-1-b). */
static int orc_step_opens(int b, int n_bins, int s) { return (s % (1 << (n_bins - 1 - b))) == 0; }

int orc_pairs_halo(int n, const double* px, const double* py, const double* pz,
                   const double* vx, const double* vy, const double* vz,
                   const uint32_t* ids, const double* h, int mode,
                   int xs_kind, double s0, double w, double mass, double dt,
                   uint64_t seed, uint64_t step, uint32_t halo,
                   orc_event* ev_out, int64_t ev_cap, orc_pair_stats* st, double* sum_p_out,
                   const uint8_t* pair_mask, const int* bins, int n_bins, int substep, double dt_max,
                   int angular)
{
    orc_geom g; memset(&g, 0, sizeof(g));
    if (mode == 0) geom_build(&g, n, px, py, pz);
    orc_kdtree T;
    kd_build(&T, n, px, py, pz, h);
    const double absmargin = mode == 0 ? ldexp(1.0, g.E + 1 - 20) : 0.0;
    double* sump = (double*)calloc((size_t)(n ? n : 1), sizeof(double));
    int64_t n_pairs = 0, n_gt1 = 0, n_near = 0, n_ev = 0;
    int overflow = 0;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    #pragma omp parallel reduction(+:n_pairs, n_gt1, n_near)
    {
        #pragma omp for schedule(dynamic, 64)
        for (int q = 0; q < n; ++q) {
            /* every pair is met from both ends; it is taken from the end q
             * that is in the mask with the other end either outside it or
             * of a larger index (no mask: the larger index) */
            if (pair_mask && !pair_mask[q]) continue;
            const double xq[3] = {px[q], py[q], pz[q]};
            int stack[128], sp = 0;
            if (T.nnode > 0) stack[sp++] = 0;
            while (sp > 0) {
                const orc_kdnode* nd = &T.node[stack[--sp]];
                const double lim = (h[q] + nd->hmax) * (1.0 + 1e-5) + absmargin;
                if (kd_box_d2(nd, xq) > lim * lim) continue;
                if (nd->left >= 0) { stack[sp++] = nd->left; stack[sp++] = nd->right; continue; }
                for (int t = nd->start; t < nd->start + nd->count; ++t) {
                    const int o = T.items[t];
                    if (o == q) continue;
                    if ((!pair_mask || pair_mask[o]) && o < q) continue;
                    const int i = (h[q] > h[o] || (h[q] == h[o] && q < o)) ? q : o;
                    const int j = i == q ? o : q;
                    /* individual steps: only pairs whose particles both start a step at
                     * this sub-step, on the longer of the two steps */
                    double dtp = dt;
                    if (bins) {
                        if (!orc_step_opens(bins[i], n_bins, substep) || !orc_step_opens(bins[j], n_bins, substep))
                            continue;
                        dtp = ldexp(dt_max, -(bins[i] < bins[j] ? bins[i] : bins[j]));
                    }
                    int inr;
                    if (mode == 0) {
                        int Ai = (int)(g.rank[i] / ORC_LEAF), Aj = (int)(g.rank[j] / ORC_LEAF);
                        float d2 = Ai <= Aj ? d2_mixed(&g, (uint32_t)i, (uint32_t)j)
                                            : d2_mixed(&g, (uint32_t)j, (uint32_t)i);
                        volatile float hs = (float)h[i] + (float)h[j];
                        volatile float lim2 = hs * hs;
                        inr = d2 < lim2;
                    } else {
                        double hs = h[i] + h[j];
                        inr = d2_fp64(px, py, pz, (uint32_t)i, (uint32_t)j) < hs * hs;
                    }
                    if (!inr) continue;
                    n_pairs++;
                    double dx = px[j] - px[i], dy = py[j] - py[i], dz = pz[j] - pz[i];
                    double d = sqrt(dx * dx + dy * dy + dz * dz);
                    double lam = orc_lambda(d, h[i], h[j]);
                    double ux = vx[i] - vx[j], uy = vy[i] - vy[j], uz = vz[i] - vz[j];
                    double v = sqrt(ux * ux + uy * uy + uz * uz);
                    double P = orc_sigma(xs_kind, s0, w, v) * mass * v * lam * dtp;
                    /* sums of P per particle, on individual steps scaled to dt_max (a rate) */
                    const double Psum = bins ? P * (dt_max / dtp) : P;
                    uint32_t a = ids[i] < ids[j] ? ids[i] : ids[j];
                    uint32_t b = ids[i] < ids[j] ? ids[j] : ids[i];
                    uint32_t ctr[4] = {(uint32_t)step, a, b, halo}, x[4];
                    orc_philox4x32_10(ctr, key, x);
                    double u = ldexp((double)x[0], -32);
                    if (angular) {
                        /* forward-dominated: every pair interacts; its record carries
                         * the step-start factor G = m_j Lambda dt instead of P */
                        if (P / 3.0 > 1.0) n_gt1++;
                    } else {
                        if (P > 1.0) n_gt1++;
                        if (fabs(P - u) < 1e-6) n_near++;
                    }
                    #pragma omp atomic
                    sump[i] += Psum;
                    #pragma omp atomic
                    sump[j] += Psum;
                    if (angular || u < P) {
                        int64_t slot;
                        #pragma omp atomic capture
                        slot = n_ev++;
                        if (slot < ev_cap) {
                            orc_event* e = &ev_out[slot];
                            e->key = ((uint64_t)halo << 54) | ((uint64_t)a << 27) | (uint64_t)b;
                            e->i = ids[i] < ids[j] ? (uint32_t)i : (uint32_t)j;
                            e->j = ids[i] < ids[j] ? (uint32_t)j : (uint32_t)i;
                            e->x1 = x[1]; e->x2 = x[2];
                            if (angular) { e->P = mass * lam * dtp; e->u = -1.0; }
                            else { e->P = P; e->u = u; }
                        } else {
                            #pragma omp atomic write
                            overflow = 1;
                        }
                    }
                }
            }
        }
    }
    double mx = 0.0;
    for (int i = 0; i < n; ++i) if (sump[i] > mx) mx = sump[i];
    if (sum_p_out) memcpy(sum_p_out, sump, sizeof(double) * (size_t)n);
    free(sump);
    st->n_pairs = n_pairs; st->n_events = n_ev; st->n_p_gt1 = n_gt1; st->n_near = n_near;
    st->max_sum_p = mx;
    kd_free(&T);
    if (mode == 0) geom_free(&g);
    return overflow ? -3 : 0;
}

static int cmp_event(const void* a, const void* b)
{
    uint64_t x = ((const orc_event*)a)->key, y = ((const orc_event*)b)->key;
    return (x > y) - (x < y);
}

void orc_sort_events(orc_event* ev, int64_t n) { qsort(ev, (size_t)n, sizeof(orc_event), cmp_event); }

/* ------------------------------------------------------------------------- */
/* Sequential application in ascending key order (multi-hit reading), each   */
/* event from the *current* FP64 velocities; isotropic direction in the CM   */
/* frame; pair momentum and energy conserved (Sect. 2, Sect. 5).             */
/* masses: per-particle masses m_i.  dE_out (optional) gets the per-event    */
/* change of the pair's kinetic energy (zero in exact arithmetic).           */
/* ------------------------------------------------------------------------- */
void orc_apply_events(const orc_event* ev, int64_t n_ev, const double* m,
                      double* vx, double* vy, double* vz, double* dE_out)
{
    for (int64_t e = 0; e < n_ev; ++e) {
        uint32_t i = ev[e].i, j = ev[e].j;
        double mi = m[i], mj = m[j], M = mi + mj;
        double vi[3] = {vx[i], vy[i], vz[i]}, vj[3] = {vx[j], vy[j], vz[j]};
        double vcm[3], dv2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            vcm[a] = (mi * vi[a] + mj * vj[a]) / M;
            double t = vi[a] - vj[a];
            dv2 += t * t;
        }
        double dv = sqrt(dv2);
        double ct = 2.0 * ldexp((double)ev[e].x1, -32) - 1.0;
        double st = sqrt(fmax(0.0, 1.0 - ct * ct));
        double phi = 2.0 * ORC_PI * ldexp((double)ev[e].x2, -32);
        double nh[3] = {st * cos(phi), st * sin(phi), ct};
        double e0 = 0.5 * mi * (vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2])
                  + 0.5 * mj * (vj[0] * vj[0] + vj[1] * vj[1] + vj[2] * vj[2]);
        double e1 = 0.0;
        double wi = mj / M * dv, wj = mi / M * dv;
        double ni[3], nj[3];
        for (int a = 0; a < 3; ++a) { ni[a] = vcm[a] + wi * nh[a]; nj[a] = vcm[a] - wj * nh[a]; }
        vx[i] = ni[0]; vy[i] = ni[1]; vz[i] = ni[2];
        vx[j] = nj[0]; vy[j] = nj[1]; vz[j] = nj[2];
        e1 = 0.5 * mi * (ni[0] * ni[0] + ni[1] * ni[1] + ni[2] * ni[2])
           + 0.5 * mj * (nj[0] * nj[0] + nj[1] * nj[1] + nj[2] * nj[2]);
        if (dE_out) dE_out[e] = e1 - e0;
    }
}

/* Forward-dominated (frictional) scattering of key-sorted pair records, one
 * after another from the current FP64 velocities (reading in the header).
 * ev[e].P holds G = m_j Lambda_ij dt of the step start; kind, s0, w give
 * sigma_V / m (Eq. vel_dep).  Outputs (may be NULL): the pair kinetic-energy
 * change and D of every record.  A record with D = 0 (zero cross-section,
 * equal velocities) leaves the velocities untouched. */
void orc_apply_drag(const orc_event* ev, int64_t n_ev, const double* m, int kind, double s0, double w,
                    double* vx, double* vy, double* vz, double* dE_out, double* D_out)
{
    for (int64_t e = 0; e < n_ev; ++e) {
        uint32_t i = ev[e].i, j = ev[e].j;
        double mi = m[i], mj = m[j], M = mi + mj;
        double vi[3] = {vx[i], vy[i], vz[i]}, vj[3] = {vx[j], vy[j], vz[j]};
        double vcm[3], u[3], u2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            vcm[a] = (mi * vi[a] + mj * vj[a]) / M;
            u[a] = vi[a] - vj[a];
            u2 += u[a] * u[a];
        }
        double un = sqrt(u2);
        double D = orc_sigma(kind, s0, w, un) / 3.0 * un * ev[e].P;
        if (D_out) D_out[e] = D;
        if (dE_out) dE_out[e] = 0.0;
        if (!(D > 0.0)) continue;               /* no turn (zero cross-section or equal velocities) */
        double ca = 1.0 - D, sa = D < 2.0 ? sqrt(D * (2.0 - D)) : 0.0;
        if (D >= 2.0) ca = -1.0;
        /* the turn's direction: an isotropic unit vector w (cos(theta) = 2 u_1 - 1,
         * phi = 2 pi u_2) projected onto the plane normal to u, normalised */
        double ct = 2.0 * ldexp((double)ev[e].x1, -32) - 1.0;
        double st = sqrt(fmax(0.0, 1.0 - ct * ct));
        double phi = 2.0 * ORC_PI * ldexp((double)ev[e].x2, -32);
        double wv[3] = {st * cos(phi), st * sin(phi), ct};
        double nh[3] = {u[0] / un, u[1] / un, u[2] / un};
        double wn = wv[0] * nh[0] + wv[1] * nh[1] + wv[2] * nh[2];
        double ep[3], el = 0.0;
        for (int a = 0; a < 3; ++a) { ep[a] = wv[a] - wn * nh[a]; el += ep[a] * ep[a]; }
        el = sqrt(el);
        double up[3];
        for (int a = 0; a < 3; ++a) up[a] = ca * u[a] + (el > 0.0 ? un * sa * ep[a] / el : 0.0);
        double e0 = 0.5 * mi * (vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2])
                  + 0.5 * mj * (vj[0] * vj[0] + vj[1] * vj[1] + vj[2] * vj[2]);
        double ni[3], nj[3];
        for (int a = 0; a < 3; ++a) { ni[a] = vcm[a] + mj / M * up[a]; nj[a] = vcm[a] - mi / M * up[a]; }
        vx[i] = ni[0]; vy[i] = ni[1]; vz[i] = ni[2];
        vx[j] = nj[0]; vy[j] = nj[1]; vz[j] = nj[2];
        double e1 = 0.5 * mi * (ni[0] * ni[0] + ni[1] * ni[1] + ni[2] * ni[2])
                  + 0.5 * mj * (nj[0] * nj[0] + nj[1] * nj[1] + nj[2] * nj[2]);
        if (dE_out) dE_out[e] = e1 - e0;
    }
}

/* ------------------------------------------------------------------------- */
/* Exact sums (Shewchuk's non-overlapping expansions, as in Python's fsum):  */
/* total kinetic energy 1/2 m |v|^2 and momentum m v of a set of particles.  */
/* Each term is formed in FP64 as term = (0.5*m) * (vx*vx + vy*vy + vz*vz)   */
/* (left to right, no FMA) and p = m*v; only the summation is exact.          */
/* ------------------------------------------------------------------------- */
/* ------------------------------------------------------------------------- */
/* Local diagnostics (Sect. 3.5 Eq. hDl, Sect. 3.6 Eq. knudsen_number, and    */
/* the effective cross-section of App. C, Eq. effective_cross_section).       */
/* Readings: the density is the SPH sum rho_i = m sum_{|x_j-x_i| < h_i}       */
/* W(|x_j - x_i|, h_i) over the particle's own kernel, itself included; the    */
/* 1-D velocity dispersion nu_i comes from the same kernel-weighted moments,   */
/* nu_i^2 = (<|v|^2> - |<v>|^2)/3; sigma_eff averages v^5 sigma_V(v) over the  */
/* relative-speed Maxwellian of two particles of 1-D dispersion nu,           */
/* f(v) ~ v^2 exp(-v^2/(4 nu^2)); sigma_V = sigma for isotropic scattering.    */
/* ------------------------------------------------------------------------- */
double orc_sigma_eff(int kind, double s0, double w, double nu)
{
    if (kind == 0) return s0;
    if (!(nu > 0.0)) return s0;
    /* num / den = int v^7 sigma(v) e^{-v^2/(4nu^2)} dv / int v^7 e^{-v^2/(4nu^2)} dv,
     * composite 8-point Gauss-Legendre on [0, 40 nu] (the tail beyond is e^{-400}) */
    const int panels = 400;
    const double L = 40.0 * nu, hp = L / panels;
    double num = 0.0, den = 0.0;
    for (int k = 0; k < panels; ++k) {
        const double a = k * hp, c = a + 0.5 * hp;
        for (int g = 0; g < 8; ++g) {
            const double v = c + 0.5 * hp * GL8_X[g];
            const double v2 = v * v;
            const double base = GL8_W[g] * v2 * v2 * v2 * v * exp(-v2 / (4.0 * nu * nu));
            num += base * orc_sigma(kind, s0, w, v);
            den += base;
        }
    }
    return num / den;
}

/* Per particle (local input order), FP64 distances of the FP64 positions:
 * out[0][i] rho_i, out[1][i] nu_i, out[2][i] sigma_eff/m at nu_i,
 * out[3][i] h/l by Eq. hDl with N_ngb and the particle mass m,
 * out[4][i] Kn by Eq. knudsen_number with gravitational constant G. */
int orc_local_diag(int n, const double* px, const double* py, const double* pz,
                   const double* vx, const double* vy, const double* vz, const double* h,
                   double m, int nngb, int kind, double s0, double w, double G, double* out)
{
    orc_kdtree T;
    kd_build(&T, n, px, py, pz, NULL);
    #pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        double sw = 0.0, sv[3] = {0.0, 0.0, 0.0}, sv2 = 0.0;
        const double hi = h[i];
        const double xi[3] = {px[i], py[i], pz[i]};
        int stack[128], sp = 0;
        if (T.nnode > 0) stack[sp++] = 0;
        while (sp > 0) {
            const orc_kdnode* nd = &T.node[stack[--sp]];
            if (kd_box_d2(nd, xi) >= hi * hi) continue;      /* every point of the box is >= h_i away */
            if (nd->left >= 0) { stack[sp++] = nd->left; stack[sp++] = nd->right; continue; }
            for (int t = nd->start; t < nd->start + nd->count; ++t) {
                const int j = T.items[t];
                const double dx = px[j] - px[i], dy = py[j] - py[i], dz = pz[j] - pz[i];
                const double d = sqrt(dx * dx + dy * dy + dz * dz);
                if (!(d < hi)) continue;          /* j == i contributes W(0, h_i) */
                const double wt = m * orc_kernel_w(d, hi);
                sw += wt;
                sv[0] += wt * vx[j]; sv[1] += wt * vy[j]; sv[2] += wt * vz[j];
                sv2 += wt * (vx[j] * vx[j] + vy[j] * vy[j] + vz[j] * vz[j]);
            }
        }
        const double rho = sw;
        const double mx = sv[0] / sw, my = sv[1] / sw, mz = sv[2] / sw;
        double var = (sv2 / sw - (mx * mx + my * my + mz * mz)) / 3.0;
        if (var < 0.0) var = 0.0;
        const double nu = sqrt(var);
        const double se = orc_sigma_eff(kind, s0, w, nu);
        out[i] = rho;
        out[(size_t)n + i] = nu;
        out[2 * (size_t)n + i] = se;
        out[3 * (size_t)n + i] = se * pow(rho, 2.0 / 3.0) * cbrt(3.0 * m * nngb / (ORC_PI * sqrt(2.0)));
        out[4 * (size_t)n + i] = sqrt(4.0 * ORC_PI * G / (rho * nu * nu)) / se;
    }
    kd_free(&T);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* SIDM time-step criterion (Sect. 2: a separate criterion for the self-      */
/* interactions; tau of the simulation table; Sect. 3.6: a minimum allowed    */
/* step).  Reading: the step on which the particle's expected number of       */
/* scatterings, sum_j P_ij for the step dt the sums were formed with, equals  */
/* tau: dt_i = tau dt / sum_j P_ij, raised to dt_min, capped at dt_max (a     */
/* particle without partners gets dt_max).  Power-of-two bins: the particle   */
/* takes the largest step dt_max / 2^b that does not exceed dt_i, b in        */
/* [0, n_bins - 1] (the smallest bin if even that is too long).               */
/* ------------------------------------------------------------------------- */
void orc_timestep(int n, const double* sum_p, double tau, double dt, double dt_min, double dt_max, int n_bins,
                  double* dt_out, int* bin_out)
{
    for (int i = 0; i < n; ++i) {
        double di = sum_p[i] > 0.0 ? tau * dt / sum_p[i] : dt_max;
        if (di < dt_min) di = dt_min;
        if (di > dt_max) di = dt_max;
        dt_out[i] = di;
        int b = 0;
        while (b < n_bins - 1 && ldexp(dt_max, -b) > di) ++b;
        bin_out[i] = b;
    }
}

/* ------------------------------------------------------------------------- */
/* Satellite in a fixed analytic host (Sect. 4.1: the host galaxy is an       */
/* external potential of six parts, the Eqs. for the NFW halo, the Hernquist  */
/* bulge and the Miyamoto-Nagai disks):                                      */
/*   Phi_NFW  = -4 pi G rho_s r_s^3 ln(1 + r / r_s) / r                      */
/*   Phi_Hern = -G M_H / (r + a_H)                                           */
/*   Phi_disk = -G M_d / sqrt(R^2 + (a_d + sqrt(z^2 + b_d^2))^2)             */
/* with r, R = sqrt(x^2 + y^2) and z measured from the host's centre.  The   */
/* host is passed as a flat array:                                           */
/*   [0] G, [1..3] centre, [4] rho_s, [5] r_s, [6] M_H, [7] a_H,              */
/*   [8] number of disks (0..4), then M_d, a_d, b_d of each disk.             */
/* A part with zero mass (density) is absent.  The acceleration is minus the */
/* gradient of the sum, differentiated by hand:                              */
/*   NFW:  -G M(<r) x / r^3,  M(<r) = 4 pi rho_s r_s^3 [ln(1+u) - u/(1+u)]   */
/*   Hern: -G M_H x / (r (r + a_H)^2)                                        */
/*   disk: -G M_d (x, y, z (a_d + zeta) / zeta) / D^(3/2),                   */
/*         zeta = sqrt(z^2 + b_d^2), D = R^2 + (a_d + zeta)^2.                */
/* Kick-drift-kick with individual power-of-two steps: at sub-step s a        */
/* particle of bin b gets the opening half kick dt_b / 2 when its step opens  */
/* at s (phase 0), the closing half kick after the drift of s when its step   */
/* closes at s + 1 (phase 1); dt_b = dt_max / 2^b.                            */
/* ------------------------------------------------------------------------- */
double orc_host_mass(double r, double rho_s, double r_s)
{
    const double u = r / r_s;
    return 4.0 * ORC_PI * rho_s * r_s * r_s * r_s * (log1p(u) - u / (1.0 + u));
}

double orc_host_phi(const double* host, double x, double y, double z)
{
    const double G = host[0];
    const double dx = x - host[1], dy = y - host[2], dz = z - host[3];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    double phi = 0.0;
    if (host[4] != 0.0) {
        const double k = 4.0 * ORC_PI * G * host[4] * host[5] * host[5] * host[5];
        phi += (r == 0.0) ? -k / host[5] : -k * log1p(r / host[5]) / r;
    }
    if (host[6] != 0.0) phi += -G * host[6] / (r + host[7]);
    const int nd = (int)host[8];
    for (int d = 0; d < nd; ++d) {
        const double M = host[9 + 3 * d], a = host[10 + 3 * d], b = host[11 + 3 * d];
        const double s = a + sqrt(dz * dz + b * b);
        phi += -G * M / sqrt(dx * dx + dy * dy + s * s);
    }
    return phi;
}

void orc_host_accel(const double* host, double x, double y, double z, double* acc)
{
    const double G = host[0];
    const double dx = x - host[1], dy = y - host[2], dz = z - host[3];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    double ax = 0.0, ay = 0.0, az = 0.0;
    if (r > 0.0) {
        double f = 0.0;
        if (host[4] != 0.0) f += -G * orc_host_mass(r, host[4], host[5]) / (r * r * r);
        if (host[6] != 0.0) f += -G * host[6] / (r * (r + host[7]) * (r + host[7]));
        ax += f * dx; ay += f * dy; az += f * dz;
    }
    const int nd = (int)host[8];
    for (int d = 0; d < nd; ++d) {
        const double M = host[9 + 3 * d], a = host[10 + 3 * d], b = host[11 + 3 * d];
        const double zeta = sqrt(dz * dz + b * b);
        const double D = dx * dx + dy * dy + (a + zeta) * (a + zeta);
        const double f = -G * M / (D * sqrt(D));
        ax += f * dx; ay += f * dy; az += f * dz * (a + zeta) / zeta;
    }
    acc[0] = ax; acc[1] = ay; acc[2] = az;
}

void orc_host_kick(int n, const double* px, const double* py, const double* pz, double* vx, double* vy, double* vz,
                   const int* bins, int n_bins, int substep, int phase, double dt_max, const double* host)
{
    for (int i = 0; i < n; ++i) {
        const int b = bins ? bins[i] : 0;
        const int period = 1 << (n_bins - 1 - b);
        const int due = phase == 0 ? (substep % period == 0) : ((substep + 1) % period == 0);
        if (!due) continue;
        double a[3];
        orc_host_accel(host, px[i], py[i], pz[i], a);
        const double h = 0.5 * ldexp(dt_max, -b);
        vx[i] += a[0] * h; vy[i] += a[1] * h; vz[i] += a[2] * h;
    }
}

/* Reflecting spherical boundary (Sect. 2: outward-moving particles beyond a  */
/* sphere about the halo are turned back without changing the energy).       */
/* Reading: outside radius rb and moving outwards, the velocity is mirrored  */
/* in the plane tangent to the sphere through the particle,                  */
/* v <- v - 2 (v . n) n with n the outward unit normal.                      */
void orc_reflect(int n, const double* px, const double* py, const double* pz, double* vx, double* vy, double* vz,
                 double cx, double cy, double cz, double rb)
{
    if (!(rb > 0.0)) return;
    for (int i = 0; i < n; ++i) {
        const double dx = px[i] - cx, dy = py[i] - cy, dz = pz[i] - cz;
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (!(r > rb)) continue;
        const double nx = dx / r, ny = dy / r, nz = dz / r;
        const double vn = vx[i] * nx + vy[i] * ny + vz[i] * nz;
        if (!(vn > 0.0)) continue;
        vx[i] -= 2.0 * vn * nx; vy[i] -= 2.0 * vn * ny; vz[i] -= 2.0 * vn * nz;
    }
}

typedef struct { double* p; int n, cap; } orc_xsum;

static void xsum_add(orc_xsum* s, double x)
{
    int k = 0;
    for (int t = 0; t < s->n; ++t) {
        double y = s->p[t];
        if (fabs(x) < fabs(y)) { double tmp = x; x = y; y = tmp; }
        double hi = x + y;
        double lo = y - (hi - x);
        if (lo != 0.0) s->p[k++] = lo;
        x = hi;
    }
    if (k >= s->cap) { s->cap = 2 * s->cap + 8; s->p = (double*)realloc(s->p, sizeof(double) * (size_t)s->cap); }
    s->n = k;
    s->p[s->n++] = x;
}

static double xsum_value(const orc_xsum* s)
{
    /* round the expansion to nearest (expansion components are non-overlapping) */
    if (s->n == 0) return 0.0;
    int t = s->n - 1;
    double hi = s->p[t], lo = 0.0;
    while (t > 0) {
        double x = hi, y = s->p[--t];
        hi = x + y;
        double yr = hi - x;
        lo = y - yr;
        if (lo != 0.0) break;
    }
    if (t > 0 && ((lo < 0.0 && s->p[t - 1] < 0.0) || (lo > 0.0 && s->p[t - 1] > 0.0))) {
        double y = lo * 2.0, x = hi + y, yr = x - hi;
        if (y == yr) hi = x;
    }
    return hi;
}

void orc_energy_momentum(int n, double m, const double* vx, const double* vy, const double* vz, double out[4])
{
    orc_xsum s[4];
    for (int a = 0; a < 4; ++a) { s[a].p = NULL; s[a].n = 0; s[a].cap = 0; }
    double hm = 0.5 * m;
    for (int i = 0; i < n; ++i) {
        double q = vx[i] * vx[i];
        q = q + vy[i] * vy[i];
        q = q + vz[i] * vz[i];
        xsum_add(&s[0], hm * q);
        xsum_add(&s[1], m * vx[i]);
        xsum_add(&s[2], m * vy[i]);
        xsum_add(&s[3], m * vz[i]);
    }
    for (int a = 0; a < 4; ++a) { out[a] = xsum_value(&s[a]); free(s[a].p); }
}

double orc_exact_sum(const double* x, int64_t n)
{
    orc_xsum s = {NULL, 0, 0};
    for (int64_t i = 0; i < n; ++i) xsum_add(&s, x[i]);
    double v = xsum_value(&s);
    free(s.p);
    return v;
}

/* Expose the canonical FP32 geometry for tests: sorted order, offsets, leaf
 * cells, cube exponent and origin. */
int orc_geometry(int n, const double* px, const double* py, const double* pz,
                 uint32_t* order_out, float* off_out, float* cell_out, int* E_out, double* O_out)
{
    orc_geom g;
    geom_build(&g, n, px, py, pz);
    if (order_out) memcpy(order_out, g.order, sizeof(uint32_t) * (size_t)n);
    if (off_out) memcpy(off_out, g.off, sizeof(float) * 3 * (size_t)n);
    if (cell_out) memcpy(cell_out, g.cell, sizeof(float) * 3 * (size_t)g.nleaf);
    if (E_out) *E_out = g.E;
    if (O_out) memcpy(O_out, g.O, sizeof(double) * 3);
    geom_free(&g);
    return 0;
}

/* canonical mixed d2 for a list of (i, j) local pairs (query i's frame) */
int orc_d2_mixed_pairs(int n, const double* px, const double* py, const double* pz,
                       int64_t npairs, const uint32_t* qi, const uint32_t* qj, float* d2_out)
{
    orc_geom g;
    geom_build(&g, n, px, py, pz);
    for (int64_t t = 0; t < npairs; ++t) d2_out[t] = d2_mixed(&g, qi[t], qj[t]);
    geom_free(&g);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
