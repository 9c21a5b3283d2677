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

// mbarrier-completed bulk copies (the one-warp kernels' staging): one
// mbarrier per ring stage, armed with the stage's byte count, waited with a
// bound (a stuck copy ends in a status bit, not a hang)
__device__ __forceinline__ void bulk_mbar_init(unsigned bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bulk_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
// global -> shared, `bytes` (multiple of 16, both addresses 16-byte aligned),
// completing on the mbarrier
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ unsigned long long bulk_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait for the phase of the given parity: false after `limit` polls
// or 2 s, whichever comes first
__device__ __forceinline__ bool bulk_wait(unsigned bar, unsigned parity, long long limit)
{
    const unsigned long long t0 = bulk_ns();
    for (long long i = 0; i < limit; ++i) {
        unsigned ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "  selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((i & 255) == 255 && bulk_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}

// hardware reciprocal square root (approximate, flush-to-zero): the inputs
// here are at least 1e-30, so no denormal reaches it
__device__ __forceinline__ float rsqrt_hw(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// hardware square root (approximate, flush-to-zero; sqrt(0) = 0, so no
// clamp).  |grad| = sqrt(q) by it instead of q * rsqrt(max(q, 1e-30)) saves a
// min/max on the ALU pipe and a multiply per point: batch of 256 grids
// 594 -> 602 GLUPS, local scheme 45.1 -> 46.8, 512^3 sphere union 469.5 ->
// 470.8 (A/B on one box)
__device__ __forceinline__ float sqrt_hw(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
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
// |grad| = sqrt(q) with the hardware square root.
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
    const float g = sqrt_hw(q);
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

// ------------------------------------------------- local scheme, FP32 ----
// Eq. 7 at a = |phi|, branch-free: with s = (a - beta)/(gamma - beta) the
// cubic is 1 - 3 s^2 + 2 s^3 (the paper's (a-gamma)^2 (2a + gamma - 3 beta)
// / (gamma - beta)^3 expanded), s clamped to [0, 1].  The end at gamma is
// tested against the smallest float >= gamma (rounded outward on the host),
// so it decides exactly as the FP64 comparison does.  The end at beta needs
// no test: every a <= beta (at most the largest float <= beta, which is at
// most the nearest float beta_n) gives a - beta_n <= 0, s = 0 and c = 1
// exactly.
__device__ __forceinline__ float cut32(float a, const LocalParams& lp)
{
    const float s = __saturatef((a - lp.beta_n) * lp.inv_w);
    const float c = fmaf(s * s, fmaf(2.f, s, -3.f), 1.f);
    return a < lp.gamma_up ? c : 0.f;
}

// Eq. 11 for the thread's four points: bit j set when point j or one of its
// face neighbours inside the domain is in T (|phi| < gamma, FP64-exact
// test), i.e. when the minimum of those |phi| is below gamma.  FACES: mask
// the neighbours beyond the domain faces.
template <bool FACES>
__device__ __forceinline__ unsigned n_nibble(const float4& c, float xm0, float xp3, const float4& ym,
                                             const float4& yp, const float4& zm, const float4& zp,
                                             bool xlo, bool xhi, bool ylo, bool yhi, bool zlo,
                                             bool zhi, float g)
{
    const float inf = __int_as_float(0x7f800000);
    float a0 = fabsf(xm0), a5 = fabsf(xp3);
    float4 Ym = ym, Yp = yp, Zm = zm, Zp = zp;
    if (FACES) {
        a0 = xlo ? inf : a0;
        a5 = xhi ? inf : a5;
        if (ylo) Ym = make_float4(inf, inf, inf, inf);
        if (yhi) Yp = make_float4(inf, inf, inf, inf);
        if (zlo) Zm = make_float4(inf, inf, inf, inf);
        if (zhi) Zp = make_float4(inf, inf, inf, inf);
    }
    const float a1 = fabsf(c.x), a2 = fabsf(c.y), a3 = fabsf(c.z), a4 = fabsf(c.w);
    const float p0 = fminf(a0, a1), p1 = fminf(a1, a2), p2 = fminf(a2, a3), p3 = fminf(a3, a4),
                p4 = fminf(a4, a5);
    const float px[4] = {fminf(p0, p1), fminf(p1, p2), fminf(p2, p3), fminf(p3, p4)};
    unsigned nb = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float yz = fminf(fminf(fabsf(comp(Ym, j)), fabsf(comp(Yp, j))),
                               fminf(fabsf(comp(Zm, j)), fabsf(comp(Zp, j))));
        nb |= (fminf(px[j], yz) < g ? 1u : 0u) << j;
    }
    return nb;
}

// One pseudo-time iteration of Eq. 12 at the thread's four points (those
// with their N bit set; the others keep their value): the upwind gradient of
// Eq. 4 where d > 0 and of Eq. 5 where d < 0, S = d / sqrt(d^2 + |Dd|^2 h^2)
// (Eq. 13) with unscaled differences (|Dd| h = sqrt(q)), then
// d - dtau S (|grad d| - 1); CLAMP: Eq. 10 afterwards, to +-(smallest float
// >= gamma), so that a clamped value stays outside T as in FP64.
// SGN = +1 / -1: every N point of the warp has its sign bit clear / set
// (d >= +0 / d <= -0; a zero gets S = 0 and keeps its value on any path);
// SGN = 0: per point, through G-(d) = G+(-d).
template <int SGN, bool FACES, bool CLAMP>
__device__ __forceinline__ float4 rei4(const float4& c, float xm0, float xp3, const float4& ym,
                                       const float4& yp, const float4& zm, const float4& zp,
                                       unsigned nb, const LocalParams& lp, bool extrap, bool xlo,
                                       bool xhi, bool ylo, bool yhi, bool zlo, bool zhi)
{
    const float xs[6] = {xm0, c.x, c.y, c.z, c.w, xp3};
    float r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float d = xs[j + 1];
        float dmx = d - xs[j], dpx = xs[j + 2] - d;
        float dmy = d - comp(ym, j), dpy = comp(yp, j) - d;
        float dmz = d - comp(zm, j), dpz = comp(zp, j) - d;
        if (FACES) {
            if (j == 0 && xlo) dmx = extrap ? dpx : 0.f;
            if (j == 3 && xhi) dpx = extrap ? dmx : 0.f;
            if (ylo) dmy = extrap ? dpy : 0.f;
            if (yhi) dpy = extrap ? dmy : 0.f;
            if (zlo) dmz = extrap ? dpz : 0.f;
            if (zhi) dpz = extrap ? dmz : 0.f;
        }
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
            const float s = d > 0.f ? 1.f : -1.f;
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
        const float gu = sqrt_hw(q);
        // d^2 + q + 1e-30 >= 1e-30 (the guard as an add on the FMA pipe
        // rather than a max on the ALU pipe, which this pass keeps busy:
        // 37.14 -> 36.79 us per pass; the two agree once d^2 + q > 2e-23)
        const float S = d * rsqrt_hw(fmaf(d, d, q + 1e-30f));
        float v = fmaf(-S, fmaf(lp.lam, gu, -lp.dtau_f), d);
        if (CLAMP) v = fminf(fmaxf(v, -lp.gamma_up), lp.gamma_up);
        r[j] = ((nb >> j) & 1u) ? v : d;
    }
    return make_float4(r[0], r[1], r[2], r[3]);
}

// the reinitialisation pass for one tile: warps without N points copy, warps
// whose N points share one sign take the sign-specialised path
template <bool FACES, bool CLAMP>
__device__ __forceinline__ float4 rei_tile(const float4& c, float xm0, float xp3, const float4& ym,
                                           const float4& yp, const float4& zm, const float4& zp,
                                           unsigned nb, const LocalParams& lp, bool extrap,
                                           bool xlo, bool xhi, bool ylo, bool yhi, bool zlo,
                                           bool zhi)
{
    if (!__any_sync(0xffffffffu, nb != 0u)) return c;
    // the sign bytes of the four values gathered into one word, and the N
    // bits spread to the sign bit of each byte (the multiplies run on the
    // FMA pipe; the float compares they replace kept the ALU pipe, which
    // bounds this pass, busier: 36.8 -> 35.5 us per pass).  A zero takes the
    // path of its sign bit; either path gives it S = 0.
    const unsigned sb = __byte_perm(__byte_perm(__float_as_uint(c.x), __float_as_uint(c.y), 0x0073),
                                    __byte_perm(__float_as_uint(c.z), __float_as_uint(c.w), 0x0073), 0x5410);
    const unsigned nbm = ((nb * 0x00204081u) & 0x01010101u) * 0x80u;
    if (__all_sync(0xffffffffu, (sb & nbm) == 0u))
        return rei4<1, FACES, CLAMP>(c, xm0, xp3, ym, yp, zm, zp, nb, lp, extrap, xlo, xhi, ylo,
                                     yhi, zlo, zhi);
    if (__all_sync(0xffffffffu, (~sb & nbm) == 0u))
        return rei4<-1, FACES, CLAMP>(c, xm0, xp3, ym, yp, zm, zp, nb, lp, extrap, xlo, xhi, ylo,
                                      yhi, zlo, zhi);
    return rei4<0, FACES, CLAMP>(c, xm0, xp3, ym, yp, zm, zp, nb, lp, extrap, xlo, xhi, ylo, yhi,
                                 zlo, zhi);
}

// N points that fall in inactive tiles: points of T on a face of this tile
// whose face neighbour tile (bits `inact`: inside the domain, not active)
// takes no part in the step, counted once per (point, face).  Zero while
// the active tiles cover N (the tiled step then equals the pointwise one).
__device__ __forceinline__ void count_breaches(const StepArgs& a, const float4& c, unsigned inact,
                                               int xh, int ly, int lz)
{
    const float g = a.lp.gamma_up;
    const unsigned tb = (fabsf(c.x) < g ? 1u : 0u) | (fabsf(c.y) < g ? 2u : 0u) |
                        (fabsf(c.z) < g ? 4u : 0u) | (fabsf(c.w) < g ? 8u : 0u);
    const unsigned nt = __popc(tb);
    unsigned bad = 0;
    if (xh == 0 && (tb & 1u) && (inact & NB_XM)) bad += 1;
    if (xh == 1 && (tb & 8u) && (inact & NB_XP)) bad += 1;
    if (ly == 0 && (inact & NB_YM)) bad += nt;
    if (ly == 7 && (inact & NB_YP)) bad += nt;
    if (lz == 0 && (inact & NB_ZM)) bad += nt;
    if (lz == 7 && (inact & NB_ZP)) bad += nt;
    if (bad && a.breaches) atomicAdd(a.breaches, (unsigned long long)bad);
}

}  // namespace lsk
