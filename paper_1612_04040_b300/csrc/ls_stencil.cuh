// ls_stencil.cuh -- device helpers shared by the FP32 stencil kernels
// (one step per pass in ls_step.cu, two steps per pass in ls_step2.cu): the
// cp.async staging primitives, programmatic dependent launch, and the
// per-point arithmetic of Eq. 3-5, so that every kernel computes the same
// bits for a point.
#pragma once

#include "ls_internal.cuh"

namespace lsk {

// cp.async of 16 / 8 / 4 bytes into shared memory at a precomputed shared
// address; when pred is false the instruction is not executed, so the global
// address is never dereferenced
__device__ __forceinline__ void cp_async16s(unsigned s, const void* gmem, bool pred = true)
{
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %2, 0;\n"
        "  @p cp.async.cg.shared.global [%0], [%1], 16; }\n" ::"r"(s), "l"(gmem), "r"((int)pred)
        : "memory");
}
__device__ __forceinline__ void cp_async8s(unsigned s, const void* gmem, bool pred = true)
{
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %2, 0;\n"
        "  @p cp.async.ca.shared.global [%0], [%1], 8; }\n" ::"r"(s), "l"(gmem), "r"((int)pred)
        : "memory");
}
__device__ __forceinline__ void cp_async4s(unsigned s, const void* gmem, bool pred = true)
{
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %2, 0;\n"
        "  @p cp.async.ca.shared.global [%0], [%1], 4; }\n" ::"r"(s), "l"(gmem), "r"((int)pred)
        : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// hardware reciprocal square root (approximate, flush-to-zero): the inputs
// here are clamped to >= 1e-30, so no denormal reaches it
__device__ __forceinline__ float rsqrt_hw(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Programmatic dependent launch: a stencil launch may start while the
// previous one drains.  Every CTA lets the next grid launch at once (it can
// only take the slots this grid frees), then waits for the previous grid's
// completion and memory before it reads anything.
__device__ __forceinline__ void pdl_launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Eq. 3-5 at one point, FP32.  Differences are unscaled (1/h is folded into
// coef = dt/h).  SGN = +1: every F >= 0 here, G+ of Eq. 4; SGN = -1: every
// F < 0, G- of Eq. 5; SGN = 0: per point, through G-(phi) = G+(-phi).
// |grad| = q * rsqrt(q) (q clamped away from 0, where the product is 0).
template <int SGN>
__device__ __forceinline__ float upd32(float c, float f, float dmx, float dpx, float dmy,
                                       float dpy, float dmz, float dpz, float coef)
{
    float ax, bx, ay, by, az, bz;
    if (SGN > 0) {
        ax = fmaxf(dmx, 0.f); bx = fminf(dpx, 0.f);
        ay = fmaxf(dmy, 0.f); by = fminf(dpy, 0.f);
        az = fmaxf(dmz, 0.f); bz = fminf(dpz, 0.f);
    } else if (SGN < 0) {
        ax = fminf(dmx, 0.f); bx = fmaxf(dpx, 0.f);
        ay = fminf(dmy, 0.f); by = fmaxf(dpy, 0.f);
        az = fminf(dmz, 0.f); bz = fmaxf(dpz, 0.f);
    } else {
        const float s = (f >= 0.f) ? 1.f : -1.f;
        ax = fmaxf(s * dmx, 0.f); bx = fminf(s * dpx, 0.f);
        ay = fmaxf(s * dmy, 0.f); by = fminf(s * dpy, 0.f);
        az = fmaxf(s * dmz, 0.f); bz = fminf(s * dpz, 0.f);
    }
    float q = ax * ax;
    q = fmaf(bx, bx, q);
    q = fmaf(ay, ay, q);
    q = fmaf(by, by, q);
    q = fmaf(az, az, q);
    q = fmaf(bz, bz, q);
    const float g = q * rsqrt_hw(fmaxf(q, 1e-30f));
    return fmaf(-(coef * f), g, c);
}

__device__ __forceinline__ float comp(const float4& v, int j)
{
    return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

// the four points of one thread.  FACES: apply the domain-face rule (only
// for tiles that touch the domain boundary).
template <int SGN, bool FACES>
__device__ __forceinline__ float4 upd4(const float4& c, const float4& f, float xm0, float xp3,
                                       const float4& ym, const float4& yp, const float4& zm,
                                       const float4& zp, float coef, bool extrap, bool xlo,
                                       bool xhi, bool ylo, bool yhi, bool zlo, bool zhi)
{
    const float xs[6] = {xm0, c.x, c.y, c.z, c.w, xp3};
    float r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float cj = xs[j + 1];
        float dmx = cj - xs[j], dpx = xs[j + 2] - cj;
        float dmy = cj - comp(ym, j), dpy = comp(yp, j) - cj;
        float dmz = cj - comp(zm, j), dpz = comp(zp, j) - cj;
        if (FACES) {
            if (j == 0 && xlo) dmx = extrap ? dpx : 0.f;
            if (j == 3 && xhi) dpx = extrap ? dmx : 0.f;
            if (ylo) dmy = extrap ? dpy : 0.f;
            if (yhi) dpy = extrap ? dmy : 0.f;
            if (zlo) dmz = extrap ? dpz : 0.f;
            if (zhi) dpz = extrap ? dmz : 0.f;
        }
        r[j] = upd32<SGN>(cj, comp(f, j), dmx, dpx, dmy, dpy, dmz, dpz, coef);
    }
    return make_float4(r[0], r[1], r[2], r[3]);
}

}  // namespace lsk
