// ls_learned.cu -- the learned coarse-grid corrector's non-convolution
// kernels (not in the paper): feature assembly, loss and its gradient, Adam,
// the band-residual check with plain-step fallback, and the fine -> coarse
// restriction.  (The convolutions and their gradients are in ls_conv.cu.)
//
// Corrector: z = CNN(features), phi^{n+1} = phi~ + h * z on band points,
// where phi~ = the plain upwind step (Eq. 3) of phi^n and the features are
// [clamp(phi^n / h, +-8), F, (phi~ - phi^n) / h] (BF16, channels-last, padded
// to 16 channels).  The check rejects the correction of a step (keeping phi~)
// if any corrected band value is not finite or |h z| exceeds one plain step's
// motion dt * max|F|.
#include <cuda_bf16.h>

#include "ls_internal.cuh"

namespace lsk {

namespace {

__device__ __forceinline__ size_t rm_index(int x, int y, int z, int nx, int ny)
{
    return ((size_t)z * ny + y) * nx + x;
}

// row-major features from row-major phi^n, phi~ and F (field or constant)
__global__ void k_features(const float* __restrict__ phi, const float* __restrict__ phit,
                           const float* __restrict__ F, float Fc, float inv_h, long long n,
                           __nv_bfloat16* __restrict__ X)
{
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const float a = phi[p];
        const float f = F ? F[p] : Fc;
        const float c0 = fminf(fmaxf(a * inv_h, -8.f), 8.f);
        const float c2 = (phit[p] - a) * inv_h;
        uint4 o[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
        __nv_bfloat16* ob = reinterpret_cast<__nv_bfloat16*>(o);
        ob[0] = __float2bfloat16_rn(c0);
        ob[1] = __float2bfloat16_rn(f);
        ob[2] = __float2bfloat16_rn(c2);
        uint4* d = reinterpret_cast<uint4*>(X + p * 16);
        d[0] = o[0];
        d[1] = o[1];
    }
}

// the same features from the bricked (tile-major) phi^n, phi~ and F of a
// single grid, written row-major: one thread per point in bricked order
// (reads contiguous; writes 8 points = 256 B contiguous per x-run)
__global__ void k_features_bricked(const float* __restrict__ phi, const float* __restrict__ phit,
                                   const float* __restrict__ F, Inst in, __nv_bfloat16* __restrict__ X)
{
    const long long n = in.ntiles * TILE_PTS;
    const float inv_h = (float)in.inv_h, Fc = (float)in.Fc;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const long long t = e / TILE_PTS;
        const int r = (int)(e - t * TILE_PTS);
        const int lx = r & 7, ly = (r >> 3) & 7, lz = r >> 6;
        const int tpl = in.tnx * in.tny;
        const int tz = (int)(t / tpl), rem = (int)(t - (long long)tz * tpl);
        const int ty = rem / in.tnx, tx = rem - ty * in.tnx;
        const size_t p = rm_index(tx * 8 + lx, ty * 8 + ly, tz * 8 + lz, in.nx, in.ny);
        const float a = phi[e];
        const float f = F ? F[e] : Fc;
        const float c0 = fminf(fmaxf(a * inv_h, -8.f), 8.f);
        const float c2 = (phit[e] - a) * inv_h;
        uint4 o[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
        __nv_bfloat16* ob = reinterpret_cast<__nv_bfloat16*>(o);
        ob[0] = __float2bfloat16_rn(c0);
        ob[1] = __float2bfloat16_rn(f);
        ob[2] = __float2bfloat16_rn(c2);
        uint4* d = reinterpret_cast<uint4*>(X + p * 16);
        d[0] = o[0];
        d[1] = o[1];
    }
}

// loss = sum over masked points of (z - t)^2 / count;  dz = 2 (z - t) / count
// on masked points (channel 0 of a 16-channel BF16 gradient), 0 elsewhere.
// mask: |phi^n| < gamma (the tube of Eq. 6), compared in FP64 like the band's
// tube test.  target t = (phi_ref - phi~) / h.
__global__ void k_loss_grad(const float* __restrict__ z, const float* __restrict__ phi,
                            const float* __restrict__ phit, const float* __restrict__ phiref,
                            float inv_h, double gamma, const int* __restrict__ count, long long n,
                            __nv_bfloat16* __restrict__ dz, double* loss)
{
    double local = 0.0;
    const float inv_cnt = 1.f / fmaxf((float)*count, 1.f);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        float g = 0.f;
        if (fabs((double)phi[p]) < gamma) {
            const float t = (phiref[p] - phit[p]) * inv_h;
            const float r = z[p] - t;
            local += (double)r * r * inv_cnt;
            g = 2.f * r * inv_cnt;
        }
        uint4 o[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
        reinterpret_cast<__nv_bfloat16*>(o)[0] = __float2bfloat16_rn(g);
        uint4* d = reinterpret_cast<uint4*>(dz + p * 16);
        d[0] = o[0];
        d[1] = o[1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local != 0.0) atomicAdd(loss, local);
}

__global__ void k_count_mask(const float* __restrict__ phi, double gamma, long long n, int* count)
{
    int local = 0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        local += fabs((double)phi[p]) < gamma;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

// Adam (bias-corrected moments) on a flat parameter vector.  The factors
// come from the host, computed in FP64 and rounded once: 1 - beta2 taken in
// FP32 from a rounded beta2 would be off by 1.3e-5 relative.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float omb1,
                       float omb2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + omb1 * gi;
    const float vi = b2 * v[i] + omb2 * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// band-residual check: over the points of active tiles, flag[0] |= the
// corrected value h z is not finite or exceeds bound = dt * M (one plain
// step's motion).  phit is bricked; z is row-major.
__global__ void k_residual_check(const float* __restrict__ z, const int* __restrict__ list,
                                 const int* __restrict__ count, Inst in, const StepScalars* sc,
                                 float hc, unsigned* flag)
{
    const int n = *count;
    const double bound = sc->dt * sc->M;
    const int tid = threadIdx.x;
    const int lx = tid & 7, ly = (tid >> 3) & 7, lz0 = tid >> 6;  // 128 threads, 2 z per pass
    bool bad = false;
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int t = list[k];
        const int tpl = in.tnx * in.tny;
        const int tz = t / tpl, r = t - tz * tpl, ty = r / in.tnx, tx = r - ty * in.tnx;
        for (int lz = lz0; lz < 8; lz += 2) {
            const float c = hc * z[rm_index(tx * 8 + lx, ty * 8 + ly, tz * 8 + lz, in.nx, in.ny)];
            if (!isfinite(c) || fabs((double)c) > bound) bad = true;
        }
    }
    if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicOr(flag, 1u);
}

// apply phi~ += h z on the active tiles unless the check failed; count the
// fallbacks (flag is cleared by the last block of the next check round)
__global__ void k_residual_apply(float* __restrict__ phit, const float* __restrict__ z,
                                 const int* __restrict__ list, const int* __restrict__ count,
                                 Inst in, float hc, const unsigned* flag)
{
    if (*flag) return;
    const int n = *count;
    const int tid = threadIdx.x;
    const int lx = tid & 7, ly = (tid >> 3) & 7, lz0 = tid >> 6;
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int t = list[k];
        const int tpl = in.tnx * in.tny;
        const int tz = t / tpl, r = t - tz * tpl, ty = r / in.tnx, tx = r - ty * in.tnx;
        for (int lz = lz0; lz < 8; lz += 2) {
            const float c = hc * z[rm_index(tx * 8 + lx, ty * 8 + ly, tz * 8 + lz, in.nx, in.ny)];
            phit[(size_t)t * TILE_PTS + (lz * 8 + ly) * 8 + lx] += c;
        }
    }
}

__global__ void k_flag_account(unsigned* flag, unsigned long long* fallbacks)
{
    if (*flag) atomicAdd(fallbacks, 1ull);
    *flag = 0;
}

// fine (row-major) -> coarse (row-major), factor 4: mean of the fine points
// 4I+1, 4I+2 per axis (the trilinear value at the coarse cell centre)
__global__ void k_restrict4(const float* __restrict__ fine, int nfx, int nfy, int nfz,
                            float* __restrict__ coarse)
{
    const int ncx = nfx / 4, ncy = nfy / 4, ncz = nfz / 4;
    const long long n = (long long)ncx * ncy * ncz;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(p % ncx), Y = (int)((p / ncx) % ncy), Z = (int)(p / ((long long)ncx * ncy));
        float s = 0.f;
        for (int k = 1; k <= 2; ++k)
            for (int j = 1; j <= 2; ++j)
                for (int i = 1; i <= 2; ++i)
                    s += fine[rm_index(4 * X + i, 4 * Y + j, 4 * Z + k, nfx, nfy)];
        coarse[p] = s * 0.125f;
    }
}

// the corrected step needs the network's output only on the active tiles;
// four 3x3x3 layers reach 4 cells, so computing every layer on the blocks
// within one tile (8 cells) of an active tile leaves those outputs exact.
// A block (bx, by, bz) of 8 x 16 x 4 points lies in tiles (bx, 2 by ..
// 2 by + 1, bz / 2).
__global__ void k_block_list(const uint8_t* __restrict__ act, Inst in, int* list, int* count)
{
    const int nbx = in.tnx, nby = in.tny / 2, nbz = 2 * in.tnz;
    const int n = nbx * nby * nbz;
    for (int blk = blockIdx.x * blockDim.x + threadIdx.x; blk < n; blk += gridDim.x * blockDim.x) {
        const int bx = blk % nbx, by = (blk / nbx) % nby, bz = blk / (nbx * nby);
        bool need = false;
        for (int tz = bz / 2 - 1; tz <= bz / 2 + 1 && !need; ++tz) {
            if (tz < 0 || tz >= in.tnz) continue;
            for (int ty = 2 * by - 1; ty <= 2 * by + 2 && !need; ++ty) {
                if (ty < 0 || ty >= in.tny) continue;
                for (int tx = bx - 1; tx <= bx + 1; ++tx) {
                    if (tx < 0 || tx >= in.tnx) continue;
                    if (act[((size_t)tz * in.tny + ty) * in.tnx + tx] & 1) {
                        need = true;
                        break;
                    }
                }
            }
        }
        if (need) list[atomicAdd(count, 1)] = blk;
    }
}

int grid_for(long long n, int threads)
{
    long long g = (n + threads - 1) / threads;
    if (g > 148 * 16) g = 148 * 16;
    return (int)(g > 0 ? g : 1);
}

}  // namespace

cudaError_t launch_features(const float* phi, const float* phit, const float* F, float Fc,
                            float inv_h, long long n, void* X, cudaStream_t s)
{
    k_features<<<grid_for(n, 256), 256, 0, s>>>(phi, phit, F, Fc, inv_h, n, (__nv_bfloat16*)X);
    return cudaGetLastError();
}

cudaError_t launch_features_bricked(const float* phi, const float* phit, const float* F,
                                   const Inst& in, void* X, cudaStream_t s)
{
    k_features_bricked<<<grid_for(in.ntiles * TILE_PTS, 256), 256, 0, s>>>(phi, phit, F, in,
                                                                          (__nv_bfloat16*)X);
    return cudaGetLastError();
}

cudaError_t launch_count_mask(const float* phi, double gamma, long long n, int* count, cudaStream_t s)
{
    k_count_mask<<<grid_for(n, 256), 256, 0, s>>>(phi, gamma, n, count);
    return cudaGetLastError();
}

cudaError_t launch_loss_grad(const float* z, const float* phi, const float* phit,
                             const float* phiref, float inv_h, double gamma, const int* count,
                             long long n, void* dz, double* loss, cudaStream_t s)
{
    k_loss_grad<<<grid_for(n, 256), 256, 0, s>>>(z, phi, phit, phiref, inv_h, gamma, count, n,
                                                 (__nv_bfloat16*)dz, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* w, const float* g, float* m, float* v, int n, float lr, int step,
                        cudaStream_t s)
{
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - pow(b1, (double)step)), c2 = (float)(1.0 - pow(b2, (double)step));
    k_adam<<<(n + 255) / 256, 256, 0, s>>>(w, g, m, v, n, lr, (float)b1, (float)b2, (float)(1.0 - b1),
                                           (float)(1.0 - b2), 1e-8f, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_residual(float* phit, const float* z, const int* list, const int* count,
                            const Inst& in, const StepScalars* sc, float hc, unsigned* flag,
                            unsigned long long* fallbacks, cudaStream_t s)
{
    const int g = 148 * 8;
    k_residual_check<<<g, 128, 0, s>>>(z, list, count, in, sc, hc, flag);
    k_residual_apply<<<g, 128, 0, s>>>(phit, z, list, count, in, hc, flag);
    k_flag_account<<<1, 1, 0, s>>>(flag, fallbacks);
    return cudaGetLastError();
}

cudaError_t launch_block_list(const uint8_t* act, const Inst& in, int* list, int* count,
                              cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    const int n = in.tnx * (in.tny / 2) * (2 * in.tnz);
    k_block_list<<<grid_for(n, 256), 256, 0, s>>>(act, in, list, count);
    return cudaGetLastError();
}

cudaError_t launch_restrict4(const float* fine, int nfx, int nfy, int nfz, float* coarse,
                             cudaStream_t s)
{
    const long long n = (long long)(nfx / 4) * (nfy / 4) * (nfz / 4);
    k_restrict4<<<grid_for(n, 256), 256, 0, s>>>(fine, nfx, nfy, nfz, coarse);
    return cudaGetLastError();
}

}  // namespace lsk
