// ls_step.cu -- the upwind step (Eq. 3-5 of section 1) on the active 8^3
// tiles of the narrow band (section 1.1, Step 2).
//
// Work decomposition: a persistent grid of 128-thread CTAs walks the active
// tile list; each CTA updates one tile per iteration.  Thread t owns the four
// x-consecutive points at (lz, ly, 4*xh..4*xh+3) = element offset 4t of the
// bricked tile, so the tile's centre values and speeds are single 16-byte
// coalesced loads.  Neighbours inside the tile come from shared memory
// (y, z) or a lane shuffle (x); the six face halos are read straight from the
// neighbouring tiles (256-byte runs for z, 32-byte runs for y, 4-byte values
// for x), which are mostly L2 hits because the active list is in ascending
// tile order.  Inactive tiles are never written (their values are frozen
// and identical in both ping-pong buffers).
//
// FP32 path: differences are taken unscaled and 1/h folded into
// coef = dt/h; the sign of F selects G+ (Eq. 4) or G- (Eq. 5) through
// G-(phi) = G+(-phi), i.e. the one-sided differences are multiplied by
// sign(F).  FP64 path: every operation of the reference definition in the
// same order with explicit round-to-nearest intrinsics (no contraction), so
// it reproduces an FP64 CPU evaluation of the definition bit for bit.
//
// Optionally (CLASSIFY) the kernel also evaluates the tube test of Eq. 6 on
// the values it has just written: min |phi^{n+1}| over the tile < gamma in
// FP64.  That saves the rebuild a full re-read of the active tiles.
#include "ls_internal.cuh"

namespace lsk {

namespace {

__device__ __forceinline__ void tile_coords(int t, const Inst& in, int& tx, int& ty, int& tz)
{
    const int tpl = in.tnx * in.tny;
    tz = t / tpl;
    const int r = t - tz * tpl;
    ty = r / in.tnx;
    tx = r - ty * in.tnx;
}

// ------------------------------------------------------------------ FP32 ----
__device__ __forceinline__ float upd32(float c, float f, float dmx, float dpx, float dmy,
                                       float dpy, float dmz, float dpz, float coef)
{
    const float s = (f >= 0.f) ? 1.f : -1.f;  // G+ for F >= 0, G- = G+(-phi) for F < 0
    const float ax = fmaxf(s * dmx, 0.f), bx = fminf(s * dpx, 0.f);
    const float ay = fmaxf(s * dmy, 0.f), by = fminf(s * dpy, 0.f);
    const float az = fmaxf(s * dmz, 0.f), bz = fminf(s * dpz, 0.f);
    float q = ax * ax;
    q = fmaf(bx, bx, q);
    q = fmaf(ay, ay, q);
    q = fmaf(by, by, q);
    q = fmaf(az, az, q);
    q = fmaf(bz, bz, q);
    const float g = sqrtf(q);
    return fmaf(-(coef * f), g, c);
}

template <bool FIELD, bool CLASSIFY>
__global__ void __launch_bounds__(128, 8) k_step_f32(StepArgs a)
{
    __shared__ float4 sm[2][8][8][2];
    __shared__ unsigned smin[2];
    const int tid = threadIdx.x;
    const int xh = tid & 1, ly = (tid >> 1) & 7, lz = tid >> 4;
    const Inst in = a.in;
    const long long n = a.list ? (long long)(*a.count) : a.fixed_count;
    if (blockIdx.x == 0 && tid == 0 && a.updates)
        atomicAdd(a.updates, (unsigned long long)n * TILE_PTS);
    const float coef = a.sc->coef;
    const float* __restrict__ src = (const float*)a.src;
    float* __restrict__ dst = (float*)a.dst;
    const float* __restrict__ Fp = (const float*)a.F;
    const float Fc = (float)in.Fc;
    const bool extrap = in.bc == 0;
    const long long sy = (long long)in.tnx * TILE_PTS;
    const long long sz = (long long)in.tnx * in.tny * TILE_PTS;
    const int off = tid * 4;
    int buf = 0;
    int prev_t = -1;
    for (long long k = blockIdx.x; k < n; k += gridDim.x) {
        const int t = a.list ? __ldg(a.list + k) : (int)k;
        int tx, ty, tz;
        tile_coords(t, in, tx, ty, tz);
        const float* tp = src + (size_t)t * TILE_PTS;
        const float4 c = __ldg(reinterpret_cast<const float4*>(tp + off));
        float4 f;
        if (FIELD) f = __ldg(reinterpret_cast<const float4*>(Fp + (size_t)t * TILE_PTS + off));
        else f = make_float4(Fc, Fc, Fc, Fc);
        // x halo: left of point 0 (xh = 0) or right of point 3 (xh = 1)
        const bool xlo_face = (xh == 0) && (tx == 0);
        const bool xhi_face = (xh == 1) && (tx == in.tnx - 1);
        float xo = 0.f;
        if (xh == 0) {
            if (!xlo_face) xo = __ldg(tp - TILE_PTS + lz * 64 + ly * 8 + 7);
        } else {
            if (!xhi_face) xo = __ldg(tp + TILE_PTS + lz * 64 + ly * 8);
        }
        // y halo (rows ly = 0 / 7)
        const bool ylo_face = (ly == 0) && (ty == 0);
        const bool yhi_face = (ly == 7) && (ty == in.tny - 1);
        float4 yo = c;
        if (ly == 0 && !ylo_face)
            yo = __ldg(reinterpret_cast<const float4*>(tp - sy + lz * 64 + 56 + 4 * xh));
        if (ly == 7 && !yhi_face)
            yo = __ldg(reinterpret_cast<const float4*>(tp + sy + lz * 64 + 4 * xh));
        // z halo (planes lz = 0 / 7)
        const bool zlo_face = (lz == 0) && (tz == 0);
        const bool zhi_face = (lz == 7) && (tz == in.tnz - 1);
        float4 zo = c;
        if (lz == 0 && !zlo_face)
            zo = __ldg(reinterpret_cast<const float4*>(tp - sz + 448 + ly * 8 + 4 * xh));
        if (lz == 7 && !zhi_face)
            zo = __ldg(reinterpret_cast<const float4*>(tp + sz + ly * 8 + 4 * xh));

        sm[buf][lz][ly][xh] = c;
        if (CLASSIFY && tid == 0) smin[buf] = 0x7f800000u;
        __syncthreads();
        if (CLASSIFY && tid == 0 && prev_t >= 0)
            a.core[prev_t] = ((double)__uint_as_float(smin[buf ^ 1]) < in.gamma) ? 1 : 0;

        const float4 ym = (ly > 0) ? sm[buf][lz][ly - 1][xh] : yo;
        const float4 yp = (ly < 7) ? sm[buf][lz][ly + 1][xh] : yo;
        const float4 zm = (lz > 0) ? sm[buf][lz - 1][ly][xh] : zo;
        const float4 zp = (lz < 7) ? sm[buf][lz + 1][ly][xh] : zo;
        const float part = __shfl_xor_sync(0xffffffffu, xh ? c.x : c.w, 1);
        const float xm0 = xh ? part : xo;
        const float xp3 = xh ? xo : part;

        // x differences (unscaled)
        const float d0 = c.x - xm0, d1 = c.y - c.x, d2 = c.z - c.y, d3 = c.w - c.z, d4 = xp3 - c.w;
        float dmx0 = d0;
        float dpx3 = d4;
        if (xlo_face) dmx0 = extrap ? d1 : 0.f;
        if (xhi_face) dpx3 = extrap ? d3 : 0.f;
        // y / z differences with the face rule
        float4 dmy = make_float4(c.x - ym.x, c.y - ym.y, c.z - ym.z, c.w - ym.w);
        float4 dpy = make_float4(yp.x - c.x, yp.y - c.y, yp.z - c.z, yp.w - c.w);
        float4 dmz = make_float4(c.x - zm.x, c.y - zm.y, c.z - zm.z, c.w - zm.w);
        float4 dpz = make_float4(zp.x - c.x, zp.y - c.y, zp.z - c.z, zp.w - c.w);
        if (ylo_face) dmy = extrap ? dpy : make_float4(0.f, 0.f, 0.f, 0.f);
        if (yhi_face) dpy = extrap ? dmy : make_float4(0.f, 0.f, 0.f, 0.f);
        if (zlo_face) dmz = extrap ? dpz : make_float4(0.f, 0.f, 0.f, 0.f);
        if (zhi_face) dpz = extrap ? dmz : make_float4(0.f, 0.f, 0.f, 0.f);

        float4 o;
        o.x = upd32(c.x, f.x, dmx0, d1, dmy.x, dpy.x, dmz.x, dpz.x, coef);
        o.y = upd32(c.y, f.y, d1, d2, dmy.y, dpy.y, dmz.y, dpz.y, coef);
        o.z = upd32(c.z, f.z, d2, d3, dmy.z, dpy.z, dmz.z, dpz.z, coef);
        o.w = upd32(c.w, f.w, d3, dpx3, dmy.w, dpy.w, dmz.w, dpz.w, coef);
        *reinterpret_cast<float4*>(dst + (size_t)t * TILE_PTS + off) = o;

        if (CLASSIFY) {
            const float m = fminf(fminf(fabsf(o.x), fabsf(o.y)), fminf(fabsf(o.z), fabsf(o.w)));
            const unsigned wm = __reduce_min_sync(0xffffffffu, __float_as_uint(m));
            if ((tid & 31) == 0) atomicMin(&smin[buf], wm);
        }
        buf ^= 1;
        prev_t = t;
    }
    if (CLASSIFY) {
        __syncthreads();
        if (tid == 0 && prev_t >= 0)
            a.core[prev_t] = ((double)__uint_as_float(smin[buf ^ 1]) < in.gamma) ? 1 : 0;
    }
}

// ------------------------------------------------------------------ FP64 ----
__device__ __forceinline__ double max0(double a) { return a > 0.0 ? a : 0.0; }
__device__ __forceinline__ double min0(double a) { return a < 0.0 ? a : 0.0; }

// one-sided difference (a - b)/h; for a power-of-two h the product with the
// exact reciprocal is the same IEEE result as the division
__device__ __forceinline__ double dq(double a, double b, bool pow2h, double h, double inv_h)
{
    const double d = __dsub_rn(a, b);
    return pow2h ? __dmul_rn(d, inv_h) : __ddiv_rn(d, h);
}

__device__ __forceinline__ double sq_sum(double a, double b)
{
    return __dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b));
}

// Eq. 3-5 in the order of the definition: per-axis sums, ((x + y) + z)
__device__ __forceinline__ double upd64(double c, double F, double dmx, double dpx, double dmy,
                                        double dpy, double dmz, double dpz, double dt)
{
    double t;
    if (F > 0.0) {
        const double sx = sq_sum(max0(dmx), min0(dpx));
        const double sy = sq_sum(max0(dmy), min0(dpy));
        const double sz = sq_sum(max0(dmz), min0(dpz));
        t = __dmul_rn(F, __dsqrt_rn(__dadd_rn(__dadd_rn(sx, sy), sz)));
    } else if (F < 0.0) {
        const double sx = sq_sum(max0(dpx), min0(dmx));
        const double sy = sq_sum(max0(dpy), min0(dmy));
        const double sz = sq_sum(max0(dpz), min0(dmz));
        // + 0.0: the inactive term max(F,0) G+ is +0, which turns a -0 into +0
        t = __dadd_rn(__dmul_rn(F, __dsqrt_rn(__dadd_rn(__dadd_rn(sx, sy), sz))), 0.0);
    } else {
        t = 0.0;
    }
    return __dsub_rn(c, __dmul_rn(dt, t));
}

struct D4 { double v[4]; };

__device__ __forceinline__ D4 ld4(const double* p)
{
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
    D4 r;
    r.v[0] = a.x; r.v[1] = a.y; r.v[2] = b.x; r.v[3] = b.y;
    return r;
}

template <bool FIELD, bool CLASSIFY>
__global__ void __launch_bounds__(128, 4) k_step_f64(StepArgs a)
{
    __shared__ D4 sm[2][8][8][2];
    __shared__ unsigned long long smin[2];
    const int tid = threadIdx.x;
    const int xh = tid & 1, ly = (tid >> 1) & 7, lz = tid >> 4;
    const Inst in = a.in;
    const long long n = a.list ? (long long)(*a.count) : a.fixed_count;
    if (blockIdx.x == 0 && tid == 0 && a.updates)
        atomicAdd(a.updates, (unsigned long long)n * TILE_PTS);
    const double dt = a.sc->dt;
    const double* __restrict__ src = (const double*)a.src;
    double* __restrict__ dst = (double*)a.dst;
    const double* __restrict__ Fp = (const double*)a.F;
    const bool extrap = in.bc == 0;
    const bool pow2h = in.pow2h != 0;
    const double h = in.h, inv_h = in.inv_h;
    const long long sy = (long long)in.tnx * TILE_PTS;
    const long long sz = (long long)in.tnx * in.tny * TILE_PTS;
    const int off = tid * 4;
    int buf = 0;
    int prev_t = -1;
    for (long long k = blockIdx.x; k < n; k += gridDim.x) {
        const int t = a.list ? __ldg(a.list + k) : (int)k;
        int tx, ty, tz;
        tile_coords(t, in, tx, ty, tz);
        const double* tp = src + (size_t)t * TILE_PTS;
        const D4 c = ld4(tp + off);
        D4 f;
        if (FIELD) f = ld4(Fp + (size_t)t * TILE_PTS + off);
        else { f.v[0] = f.v[1] = f.v[2] = f.v[3] = in.Fc; }
        const bool xlo_face = (xh == 0) && (tx == 0);
        const bool xhi_face = (xh == 1) && (tx == in.tnx - 1);
        double xo = 0.0;
        if (xh == 0) {
            if (!xlo_face) xo = __ldg(tp - TILE_PTS + lz * 64 + ly * 8 + 7);
        } else {
            if (!xhi_face) xo = __ldg(tp + TILE_PTS + lz * 64 + ly * 8);
        }
        const bool ylo_face = (ly == 0) && (ty == 0);
        const bool yhi_face = (ly == 7) && (ty == in.tny - 1);
        D4 yo = c;
        if (ly == 0 && !ylo_face) yo = ld4(tp - sy + lz * 64 + 56 + 4 * xh);
        if (ly == 7 && !yhi_face) yo = ld4(tp + sy + lz * 64 + 4 * xh);
        const bool zlo_face = (lz == 0) && (tz == 0);
        const bool zhi_face = (lz == 7) && (tz == in.tnz - 1);
        D4 zo = c;
        if (lz == 0 && !zlo_face) zo = ld4(tp - sz + 448 + ly * 8 + 4 * xh);
        if (lz == 7 && !zhi_face) zo = ld4(tp + sz + ly * 8 + 4 * xh);

        sm[buf][lz][ly][xh] = c;
        if (CLASSIFY && tid == 0) smin[buf] = 0x7ff0000000000000ull;
        __syncthreads();
        if (CLASSIFY && tid == 0 && prev_t >= 0)
            a.core[prev_t] = (__longlong_as_double((long long)smin[buf ^ 1]) < in.gamma) ? 1 : 0;

        const D4 ym = (ly > 0) ? sm[buf][lz][ly - 1][xh] : yo;
        const D4 yp = (ly < 7) ? sm[buf][lz][ly + 1][xh] : yo;
        const D4 zm = (lz > 0) ? sm[buf][lz - 1][ly][xh] : zo;
        const D4 zp = (lz < 7) ? sm[buf][lz + 1][ly][xh] : zo;
        const double part = __shfl_xor_sync(0xffffffffu, xh ? c.v[0] : c.v[3], 1);
        double xn[6];  // x values at x0-1 .. x0+4
        xn[0] = xh ? part : xo;
        xn[1] = c.v[0]; xn[2] = c.v[1]; xn[3] = c.v[2]; xn[4] = c.v[3];
        xn[5] = xh ? xo : part;

        D4 o;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const double cj = c.v[j];
            double dmx = dq(cj, xn[j], pow2h, h, inv_h);
            double dpx = dq(xn[j + 2], cj, pow2h, h, inv_h);
            double dmy = dq(cj, ym.v[j], pow2h, h, inv_h);
            double dpy = dq(yp.v[j], cj, pow2h, h, inv_h);
            double dmz = dq(cj, zm.v[j], pow2h, h, inv_h);
            double dpz = dq(zp.v[j], cj, pow2h, h, inv_h);
            if (j == 0 && xlo_face) dmx = extrap ? dpx : 0.0;
            if (j == 3 && xhi_face) dpx = extrap ? dmx : 0.0;
            if (ylo_face) dmy = extrap ? dpy : 0.0;
            if (yhi_face) dpy = extrap ? dmy : 0.0;
            if (zlo_face) dmz = extrap ? dpz : 0.0;
            if (zhi_face) dpz = extrap ? dmz : 0.0;
            o.v[j] = upd64(cj, f.v[j], dmx, dpx, dmy, dpy, dmz, dpz, dt);
        }
        double* dp = dst + (size_t)t * TILE_PTS + off;
        *reinterpret_cast<double2*>(dp) = make_double2(o.v[0], o.v[1]);
        *reinterpret_cast<double2*>(dp + 2) = make_double2(o.v[2], o.v[3]);

        if (CLASSIFY) {
            double m = fmin(fmin(fabs(o.v[0]), fabs(o.v[1])), fmin(fabs(o.v[2]), fabs(o.v[3])));
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, s));
            if ((tid & 31) == 0)
                atomicMin(&smin[buf], (unsigned long long)__double_as_longlong(m));
        }
        buf ^= 1;
        prev_t = t;
    }
    if (CLASSIFY) {
        __syncthreads();
        if (tid == 0 && prev_t >= 0)
            a.core[prev_t] = (__longlong_as_double((long long)smin[buf ^ 1]) < in.gamma) ? 1 : 0;
    }
}

template <typename K>
int occupancy_grid(K kernel)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 128, 0);
    if (per < 1) per = 1;
    return sms * per;
}

}  // namespace

int step_grid_size(int prec, int classify)
{
    static int cache[2][2] = {{0, 0}, {0, 0}};
    int& g = cache[prec ? 1 : 0][classify ? 1 : 0];
    if (!g) {
        if (prec == 0)
            g = classify ? occupancy_grid(k_step_f32<true, true>) : occupancy_grid(k_step_f32<true, false>);
        else
            g = classify ? occupancy_grid(k_step_f64<true, true>) : occupancy_grid(k_step_f64<true, false>);
    }
    return g;
}

cudaError_t launch_step(const StepArgs& a, int prec, int grid, cudaStream_t s)
{
    const bool field = a.F != nullptr;
    const bool cls = a.core != nullptr;
    if (prec == 0) {
        if (field && cls) k_step_f32<true, true><<<grid, 128, 0, s>>>(a);
        else if (field) k_step_f32<true, false><<<grid, 128, 0, s>>>(a);
        else if (cls) k_step_f32<false, true><<<grid, 128, 0, s>>>(a);
        else k_step_f32<false, false><<<grid, 128, 0, s>>>(a);
    } else {
        if (field && cls) k_step_f64<true, true><<<grid, 128, 0, s>>>(a);
        else if (field) k_step_f64<true, false><<<grid, 128, 0, s>>>(a);
        else if (cls) k_step_f64<false, true><<<grid, 128, 0, s>>>(a);
        else k_step_f64<false, false><<<grid, 128, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace lsk
