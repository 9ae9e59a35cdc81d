// sidm_static.cu -- allocation-free per-halo kinetic energy and momentum.
//
// Some callers cannot let a library allocate device memory: a plug-in inside
// a host application whose framework owns every byte of the device (its own
// caching allocator, a fixed memory budget) must not call cudaMalloc or
// cudaFree.  sidm_energy_momentum_static serves them: it needs no context and
// keeps its scratch (four double-double sums per chunk of 16384 particles)
// in a file-scope __device__ array of fixed size, which every GPU that loads
// this library holds until the process exits.
//
// The arithmetic is that of sidm_energy_momentum (sidm_sum.cuh, the same
// chunks of 16384 particles and the same per-chunk and per-halo code), so the
// result is bit-identical to the context-based call on the same inputs.
#include <mutex>
#include <string>

#include "../../include/sidm.h"
#include "sidm_sum.cuh"

namespace {

constexpr int kStaticChunk = 16384;

// Scratch of every call: [SIDM_STATIC_MAX_CHUNKS][8] chunk sums, then
// [kStaticMaxGroups][8] group sums (doubles, 268 KiB).  Each call overwrites
// the entries of its own chunks and groups before reading them, so nothing has
// to start at zero.  Calls that overlap on the GPU race here.
constexpr int kStaticMaxGroups = SIDM_STATIC_MAX_CHUNKS / sidm_sum::kGroupChunks + SIDM_STATIC_MAX_HALOS;
static __device__ __align__(256) double g_static_partials[(SIDM_STATIC_MAX_CHUNKS + kStaticMaxGroups) * 8];

struct StaticLayout {
    int n_halos;
    int n_chunks;
    int n_groups;
    long long halo_off[SIDM_STATIC_MAX_HALOS + 1];
    int chunk_off[SIDM_STATIC_MAX_HALOS + 1];   // first chunk of each halo
    int group_off[SIDM_STATIC_MAX_HALOS + 1];   // first group of chunks of each halo
};

static_assert(kStaticChunk <= sidm_sum::kMaxChunk, "chunk larger than the exact-sum windows allow");

template <class R>
__global__ void __launch_bounds__(sidm_sum::chunk_threads<R>()) k_static_partial(StaticLayout lay, const R* __restrict__ vel,
                                                                      long long N, double* __restrict__ part)
{
    const int c = blockIdx.x;
    int h = 0;
    while (h + 1 < lay.n_halos && lay.chunk_off[h + 1] <= c) ++h;
    const long long b = lay.halo_off[h] + (long long)(c - lay.chunk_off[h]) * kStaticChunk;
    long long e = b + kStaticChunk;
    if (e > lay.halo_off[h + 1]) e = lay.halo_off[h + 1];
    sidm_sum::chunk_sums(vel, N, b, e, part + 8 * (long long)c);
}

// the two merge levels of sidm_sum.cuh, in the order sidm_energy_momentum uses
__global__ void k_static_group(StaticLayout lay, const double* __restrict__ part, double* __restrict__ gpart)
{
    const int g = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);   // one warp per group
    if (g >= lay.n_groups) return;
    int h = 0;
    while (h + 1 < lay.n_halos && lay.group_off[h + 1] <= g) ++h;
    const int c0 = lay.chunk_off[h] + (g - lay.group_off[h]) * sidm_sum::kGroupChunks;
    const int c1 = min(c0 + sidm_sum::kGroupChunks, lay.chunk_off[h + 1]);
    sidm_sum::group_sums(part, c0, c1, gpart + 8 * (long long)g);
}

__global__ void k_static_final(StaticLayout lay, const double* __restrict__ mass, const double* __restrict__ gpart,
                               double* __restrict__ out, double* __restrict__ comp)
{
    const int h = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);   // one warp per halo
    if (h >= lay.n_halos) return;
    sidm_sum::halo_result(gpart, lay.group_off[h], lay.group_off[h + 1], mass[h], out + 4 * h,
                          comp ? comp + 4 * h : nullptr);
}

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
double* g_static_ptr[kMaxDevices] = {};   // address of the last lookup per device
thread_local std::string g_static_err;
int static_fail(int code, const std::string& m)
{
    g_static_err = m;
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
    lay.group_off[0] = 0;
    long long chunks = 0;
    for (int h = 0; h < n_halos; ++h) {
        if (halo_off[h + 1] < halo_off[h]) return static_fail(SIDM_EINVAL, "halo_off must be non-decreasing");
        lay.halo_off[h] = halo_off[h];
        chunks += (halo_off[h + 1] - halo_off[h] + kStaticChunk - 1) / kStaticChunk;
        if (chunks > SIDM_STATIC_MAX_CHUNKS)
            return static_fail(SIDM_ECAPACITY, "more than SIDM_STATIC_MAX_CHUNKS chunks of 16384 particles");
        lay.chunk_off[h + 1] = (int)chunks;
        const int nc = lay.chunk_off[h + 1] - lay.chunk_off[h];
        lay.group_off[h + 1] = lay.group_off[h] + (nc + sidm_sum::kGroupChunks - 1) / sidm_sum::kGroupChunks;
    }
    lay.n_groups = lay.group_off[n_halos];
    lay.halo_off[n_halos] = halo_off[n_halos];
    lay.n_chunks = (int)chunks;
    if (!mass_dev || !out_dev || (halo_off[n_halos] > 0 && !vel_dev)) return static_fail(SIDM_EINVAL, "null argument");

    // Device address of the scratch array, with this device current (host code
    // only sees a stand-in for the symbol).  Outside stream capture it is looked
    // up on every call, so a context torn down and re-created (cudaDeviceReset)
    // never leaves a stale address behind; during capture the address of the
    // last uncaptured call on this device is used.
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(SIDM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return static_fail(SIDM_EINVAL, "device ordinal out of range");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return static_fail(SIDM_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
    double* part = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (cap == cudaStreamCaptureStatusNone) {
            double* p = nullptr;
            e = cudaGetSymbolAddress((void**)&p, g_static_partials);
            if (e != cudaSuccess) {
                g_static_ptr[dev] = nullptr;
                return static_fail(SIDM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
            g_static_ptr[dev] = p;
        } else if (!g_static_ptr[dev]) {
            return static_fail(SIDM_EINVAL, "the first call on a device must come before any stream capture");
        }
        part = g_static_ptr[dev];
    }
    const long long N = halo_off[n_halos];
    if (chunks > 0) {
        if (precision == SIDM_FP64)
            k_static_partial<double><<<(unsigned)chunks, sidm_sum::chunk_threads<double>(), 0, stream>>>(lay, (const double*)vel_dev, N,
                                                                                          part);
        else
            k_static_partial<float><<<(unsigned)chunks, sidm_sum::chunk_threads<float>(), 0, stream>>>(lay, (const float*)vel_dev, N,
                                                                                         part);
        e = cudaGetLastError();
        if (e != cudaSuccess) return static_fail(SIDM_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    }
    double* gpart = part + (size_t)SIDM_STATIC_MAX_CHUNKS * 8;
    if (lay.n_groups > 0) {
        k_static_group<<<(unsigned)((lay.n_groups + 3) / 4), 128, 0, stream>>>(lay, part, gpart);
        e = cudaGetLastError();
        if (e != cudaSuccess) return static_fail(SIDM_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    }
    k_static_final<<<(n_halos + 3) / 4, 128, 0, stream>>>(lay, mass_dev, gpart, out_dev, comp_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(SIDM_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    g_static_err.clear();
    return SIDM_OK;
}

extern "C" const char* sidm_static_last_error(void) { return g_static_err.c_str(); }
