// sidm_static.cu -- allocation-free per-halo kinetic energy and momentum.
//
// Some callers cannot let a library allocate device memory: a plug-in inside
// a host application whose framework owns every byte of the device (its own
// caching allocator, a fixed memory budget) must not call cudaMalloc or
// cudaFree.  sidm_energy_momentum_static serves them: it needs no context and
// keeps its scratch (one FP64 partial sum pair per chunk of 16384 particles)
// in a file-scope __device__ array of fixed size, which every GPU that loads
// this library holds until the process exits.
//
// The arithmetic and its order are those of sidm_energy_momentum: per chunk,
// thread t sums elements t, t+256, ... with two-sum compensation, then a
// fixed binary tree over the 256 threads; per halo the chunk partials are
// merged in chunk order.  The result is therefore bit-identical to the
// context-based call on the same inputs.
#include <mutex>
#include <string>

#include "../../include/sidm.h"

namespace {

constexpr int kStaticChunk = 16384;

// Scratch of every call: [SIDM_STATIC_MAX_CHUNKS][8] doubles = 256 KiB.
// Each call overwrites the entries of its own chunks before reading them, so
// nothing has to start at zero.  Calls that overlap on the GPU race here.
static __device__ __align__(256) double g_static_partials[SIDM_STATIC_MAX_CHUNKS * 8];

struct StaticLayout {
    int n_halos;
    int n_chunks;
    long long halo_off[SIDM_STATIC_MAX_HALOS + 1];
    int chunk_off[SIDM_STATIC_MAX_HALOS + 1];   // first chunk of each halo
};

struct Comp2 { double s, c; };

__device__ __forceinline__ void two_sum2(double a, double b, double& s, double& e)
{
    s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

__device__ __forceinline__ void comp_add2(Comp2& x, double v)
{
    double s, e;
    two_sum2(x.s, v, s, e);
    x.s = s;
    x.c = __dadd_rn(x.c, e);
}

__device__ __forceinline__ void comp_merge2(Comp2& x, const Comp2& y)
{
    double s, e;
    two_sum2(x.s, y.s, s, e);
    x.s = s;
    x.c = __dadd_rn(__dadd_rn(x.c, y.c), e);
}

template <class R>
__global__ void __launch_bounds__(256) k_static_partial(StaticLayout lay, const R* __restrict__ vel, long long N,
                                                        const double* __restrict__ mass, double* __restrict__ part)
{
    __shared__ Comp2 sh[4][256];
    const int c = blockIdx.x;
    int h = 0;
    while (h + 1 < lay.n_halos && lay.chunk_off[h + 1] <= c) ++h;
    const long long b = lay.halo_off[h] + (long long)(c - lay.chunk_off[h]) * kStaticChunk;
    long long e = b + kStaticChunk;
    if (e > lay.halo_off[h + 1]) e = lay.halo_off[h + 1];
    const double m = mass[h];
    const double hm = __dmul_rn(0.5, m);
    Comp2 acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (long long s = b + threadIdx.x; s < e; s += 256) {
        const double x = (double)vel[s], y = (double)vel[N + s], z = (double)vel[2 * N + s];
        double q = __dmul_rn(x, x);
        q = __dadd_rn(q, __dmul_rn(y, y));
        q = __dadd_rn(q, __dmul_rn(z, z));
        comp_add2(acc[0], __dmul_rn(hm, q));
        comp_add2(acc[1], __dmul_rn(m, x));
        comp_add2(acc[2], __dmul_rn(m, y));
        comp_add2(acc[3], __dmul_rn(m, z));
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) sh[a][threadIdx.x] = acc[a];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int a = 0; a < 4; ++a) comp_merge2(sh[a][threadIdx.x], sh[a][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x < 4) {
        part[c * 8 + 2 * threadIdx.x] = sh[threadIdx.x][0].s;
        part[c * 8 + 2 * threadIdx.x + 1] = sh[threadIdx.x][0].c;
    }
}

__global__ void k_static_final(StaticLayout lay, const double* __restrict__ part, double* __restrict__ out,
                               double* __restrict__ comp)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= lay.n_halos) return;
    Comp2 acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int c = lay.chunk_off[h]; c < lay.chunk_off[h + 1]; ++c)
        for (int a = 0; a < 4; ++a) comp_merge2(acc[a], Comp2{part[c * 8 + 2 * a], part[c * 8 + 2 * a + 1]});
    for (int a = 0; a < 4; ++a) {
        const double v = __dadd_rn(acc[a].s, acc[a].c);
        out[h * 4 + a] = v;
        if (comp) comp[h * 4 + a] = __dsub_rn(acc[a].c, __dsub_rn(v, acc[a].s));
    }
}

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
double* g_static_ptr[kMaxDevices] = {};
int static_fail(int code, const std::string& m)
{
    (void)m;   // the return code carries the failure; the texts document each case
    return code;
}

}  // namespace

extern "C" int sidm_energy_momentum_static(int32_t n_halos, const int64_t* halo_off, int32_t precision,
                                           const double* mass_dev, const void* vel_dev, double* out_dev,
                                           double* comp_dev, cudaStream_t stream)
{
    if (n_halos < 1 || n_halos > SIDM_STATIC_MAX_HALOS || !halo_off)
        return static_fail(SIDM_EINVAL, "n_halos must be in [1, SIDM_STATIC_MAX_HALOS]");
    if (precision != SIDM_MIXED && precision != SIDM_FP64) return static_fail(SIDM_EINVAL, "bad precision");
    if (halo_off[0] != 0) return static_fail(SIDM_EINVAL, "halo_off[0] must be 0");
    StaticLayout lay;
    lay.n_halos = n_halos;
    lay.chunk_off[0] = 0;
    long long chunks = 0;
    for (int h = 0; h < n_halos; ++h) {
        if (halo_off[h + 1] < halo_off[h]) return static_fail(SIDM_EINVAL, "halo_off must be non-decreasing");
        lay.halo_off[h] = halo_off[h];
        chunks += (halo_off[h + 1] - halo_off[h] + kStaticChunk - 1) / kStaticChunk;
        if (chunks > SIDM_STATIC_MAX_CHUNKS)
            return static_fail(SIDM_ECAPACITY, "more than SIDM_STATIC_MAX_CHUNKS chunks of 16384 particles");
        lay.chunk_off[h + 1] = (int)chunks;
    }
    lay.halo_off[n_halos] = halo_off[n_halos];
    lay.n_chunks = (int)chunks;
    if (!mass_dev || !out_dev || (halo_off[n_halos] > 0 && !vel_dev)) return static_fail(SIDM_EINVAL, "null argument");

    // Device address of the scratch array, looked up once per device with
    // that device current (host code only sees a stand-in for the symbol).
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(SIDM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return static_fail(SIDM_EINVAL, "device ordinal out of range");
    double* part = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_ptr[dev]) {
            e = cudaGetSymbolAddress((void**)&g_static_ptr[dev], g_static_partials);
            if (e != cudaSuccess) {
                g_static_ptr[dev] = nullptr;
                return static_fail(SIDM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
        }
        part = g_static_ptr[dev];
    }
    const long long N = halo_off[n_halos];
    if (chunks > 0) {
        if (precision == SIDM_FP64)
            k_static_partial<double><<<(unsigned)chunks, 256, 0, stream>>>(lay, (const double*)vel_dev, N, mass_dev, part);
        else
            k_static_partial<float><<<(unsigned)chunks, 256, 0, stream>>>(lay, (const float*)vel_dev, N, mass_dev, part);
        e = cudaGetLastError();
        if (e != cudaSuccess) return static_fail(SIDM_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    }
    k_static_final<<<(n_halos + 127) / 128, 128, 0, stream>>>(lay, part, out_dev, comp_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(SIDM_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return SIDM_OK;
}
