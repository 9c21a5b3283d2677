// ls_noalloc.cu -- ls_band_tiles_noalloc: the band's active-tile list
// computed with no device allocation at all.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured by someone else, host code inside a real-time or
// allocation-free section (a simulation step that must never hit the
// allocator or its implicit synchronisation), or an embedding application
// whose memory pool owns the whole device.  This entry point serves them:
// the caller passes phi and the output buffers, and the only scratch the
// kernels need (tile flags and per-block counts) lives in one file-scope
// __device__ array of fixed size.  With CUDA's lazy module loading (the
// default) the array is reserved when this file's module is first loaded
// on a device, i.e. by the first call there (its cudaGetSymbolAddress); it
// is then held until the process exits.  A caller warms a device up with
// one throwaway call made outside any capture and allocation-free section.
//
// The kernels are separate copies of the band-rebuild steps (tube test per
// tile, 26-neighbour dilation, count, scan, ascending scatter) that read phi
// in the caller's row-major layout; the context-based path is untouched.
#include <cmath>
#include <mutex>

#include "ls.h"
#include "ls_internal.cuh"

namespace {

constexpr long long NA_MAX_TILES = LS_NOALLOC_MAX_TILES;
constexpr int NA_BLOCK = 256;
constexpr int NA_MAX_BLOCKS = (int)(NA_MAX_TILES / NA_BLOCK);
// layout of the scratch array: core flags | active flags | block counts
constexpr size_t NA_CORE_OFF = 0;
constexpr size_t NA_ACT_OFF = NA_MAX_TILES;
constexpr size_t NA_CNT_OFF = 2 * NA_MAX_TILES;
constexpr size_t NA_BYTES = NA_CNT_OFF + sizeof(int) * NA_MAX_BLOCKS;

static __device__ __align__(256) unsigned char g_na_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
void* g_na_ptr[NA_MAX_DEVICES] = {};

// device address of g_na_scratch on the current device (set up once per
// device, with that device current)
cudaError_t na_scratch(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

template <typename T>
__device__ __forceinline__ T inf_of()
{
    if constexpr (sizeof(T) == 4) return __int_as_float(0x7f800000);
    else return __longlong_as_double(0x7ff0000000000000ll);
}

// Eq. 6 per tile on a row-major grid: one warp per tile, lane -> two of the
// tile's 64 x-rows of 8 values
template <typename T>
__global__ void __launch_bounds__(256) k_na_classify(const T* __restrict__ phi, int nx, int ny,
                                                     int tnx, int tny, long long ntiles,
                                                     double gamma, uint8_t* core)
{
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * 8;
    for (long long t = (long long)blockIdx.x * 8 + (threadIdx.x >> 5); t < ntiles; t += warps) {
        const int tz = (int)(t / ((long long)tnx * tny));
        const int rem = (int)(t - (long long)tz * tnx * tny);
        const int ty = rem / tnx, tx = rem - ty * tnx;
        T m = inf_of<T>();
        for (int r = lane; r < 64; r += 32) {
            const int z = tz * 8 + (r >> 3), y = ty * 8 + (r & 7);
            const T* row = phi + ((size_t)z * ny + y) * nx + (size_t)tx * 8;
            for (int i = 0; i < 8; ++i) {
                const T v = row[i] < T(0) ? -row[i] : row[i];
                m = v < m ? v : m;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T u = __shfl_xor_sync(0xffffffffu, m, o);
            m = u < m ? u : m;
        }
        if (lane == 0) core[t] = ((double)m < gamma) ? 1 : 0;
    }
}

// one-tile dilation (26 neighbours) and per-block counts
__global__ void __launch_bounds__(NA_BLOCK) k_na_dilate(const uint8_t* __restrict__ core,
                                                        uint8_t* act, int tnx, int tny, int tnz,
                                                        long long ntiles, int* counts)
{
    const long long t = (long long)blockIdx.x * NA_BLOCK + threadIdx.x;
    int on = 0;
    if (t < ntiles) {
        const int tz = (int)(t / ((long long)tnx * tny));
        const int rem = (int)(t - (long long)tz * tnx * tny);
        const int ty = rem / tnx, tx = rem - ty * tnx;
        for (int dz = -1; dz <= 1 && !on; ++dz)
            for (int dy = -1; dy <= 1 && !on; ++dy)
                for (int dx = -1; dx <= 1 && !on; ++dx) {
                    const int x = tx + dx, y = ty + dy, z = tz + dz;
                    if (x < 0 || y < 0 || z < 0 || x >= tnx || y >= tny || z >= tnz) continue;
                    on = core[((long long)z * tny + y) * tnx + x];
                }
        act[t] = (uint8_t)on;
    }
    const int c = __syncthreads_count(on);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// exclusive scan of the block counts (one block); total -> *count_out
__global__ void __launch_bounds__(1024) k_na_scan(int* counts, int nblocks, int* count_out)
{
    __shared__ int sums[1024];
    const int per = (nblocks + 1023) / 1024;
    const int b0 = threadIdx.x * per;
    int local = 0;
    for (int k = 0; k < per; ++k)
        if (b0 + k < nblocks) local += counts[b0 + k];
    sums[threadIdx.x] = local;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = (int)threadIdx.x >= o ? sums[threadIdx.x - o] : 0;
        __syncthreads();
        sums[threadIdx.x] += v;
        __syncthreads();
    }
    int run = sums[threadIdx.x] - local;
    for (int k = 0; k < per; ++k) {
        if (b0 + k < nblocks) {
            const int c = counts[b0 + k];
            counts[b0 + k] = run;
            run += c;
        }
    }
    if (threadIdx.x == 1023) *count_out = run;
}

// ascending scatter of the active tile ids
__global__ void __launch_bounds__(NA_BLOCK) k_na_scatter(const uint8_t* __restrict__ act,
                                                         const int* __restrict__ offsets,
                                                         long long ntiles, int* ids)
{
    __shared__ int warp_cnt[NA_BLOCK / 32];
    const long long t = (long long)blockIdx.x * NA_BLOCK + threadIdx.x;
    const int on = (t < ntiles) ? act[t] : 0;
    const unsigned b = __ballot_sync(0xffffffffu, on);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) warp_cnt[w] = __popc(b);
    __syncthreads();
    int before = 0;
    for (int k = 0; k < w; ++k) before += warp_cnt[k];
    if (on) ids[offsets[blockIdx.x] + before + __popc(b & ((1u << lane) - 1u))] = (int)t;
}

// Launches one kernel and returns that launch's own status: the runtime
// call's return value, not cudaGetLastError, so an error left pending by
// the caller's earlier work is neither reported as ours nor cleared.
template <typename... P, typename... A>
cudaError_t na_launch(void (*kernel)(P...), int grid, int block, cudaStream_t s, A... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    return cudaLaunchKernelEx(&cfg, kernel, (P)args...);
}

}  // namespace

extern "C" int ls_band_tiles_noalloc(const void* phi, int nx, int ny, int nz, double h,
                                     int precision, double halfwidth_in_h, int* tiles_out,
                                     long long tiles_cap, int* count_out, void* cuda_stream)
{
    // every argument is checked on the host before the first CUDA call
    if (!phi || !tiles_out || !count_out) return LS_EINVAL;
    if (nx < 8 || ny < 8 || nz < 8 || nx % 8 || ny % 8 || nz % 8) return LS_EINVAL;
    if (!std::isfinite(h) || !(h > 0.0) || !std::isfinite(halfwidth_in_h) || !(halfwidth_in_h > 0.0))
        return LS_EINVAL;
    if (precision != LS_FP32 && precision != LS_FP64) return LS_EINVAL;
    const int tnx = nx / 8, tny = ny / 8, tnz = nz / 8;
    const long long ntiles = (long long)tnx * tny * tnz;
    if (ntiles > NA_MAX_TILES) return LS_EINVAL;  // beyond the fixed scratch size
    if (tiles_cap < ntiles) return LS_EINVAL;
    const double gamma = halfwidth_in_h * h;
    if (!std::isfinite(gamma)) return LS_EINVAL;
    void* base = nullptr;
    cudaError_t e = na_scratch(&base);
    if (e != cudaSuccess) return LS_ECUDA;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return LS_ECUDA;
    uint8_t* core = (uint8_t*)base + NA_CORE_OFF;
    uint8_t* act = (uint8_t*)base + NA_ACT_OFF;
    int* counts = (int*)((uint8_t*)base + NA_CNT_OFF);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    long long g = (ntiles + 7) / 8;  // grid-stride: 8 tiles (warps) per block
    if (g > (long long)sms * 64) g = (long long)sms * 64;
    if (precision == LS_FP32)
        e = na_launch(k_na_classify<float>, (int)g, 256, s, (const float*)phi, nx, ny, tnx, tny,
                      ntiles, gamma, core);
    else
        e = na_launch(k_na_classify<double>, (int)g, 256, s, (const double*)phi, nx, ny, tnx, tny,
                      ntiles, gamma, core);
    if (e != cudaSuccess) return LS_ECUDA;
    const int nb = (int)((ntiles + NA_BLOCK - 1) / NA_BLOCK);
    e = na_launch(k_na_dilate, nb, NA_BLOCK, s, (const uint8_t*)core, act, tnx, tny, tnz, ntiles,
                  counts);
    if (e != cudaSuccess) return LS_ECUDA;
    e = na_launch(k_na_scan, 1, 1024, s, counts, nb, count_out);
    if (e != cudaSuccess) return LS_ECUDA;
    e = na_launch(k_na_scatter, nb, NA_BLOCK, s, (const uint8_t*)act, (const int*)counts, ntiles,
                  tiles_out);
    if (e != cudaSuccess) return LS_ECUDA;
    return LS_OK;
}
