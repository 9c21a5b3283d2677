// ls_step64.cu -- the FP64 upwind step (Eq. 3-5 of section 1) and the FP64
// local-scheme passes (Eq. 8, 10, 12-13) on the active 8^3 tiles.
//
// Every operation of the definition in the same order with explicit
// round-to-nearest intrinsics (no contraction), so the result is an FP64
// CPU evaluation of the definition bit for bit.  The FP64 pipe is the
// bound on B300, so the plain step for a power-of-two h skips the six
// scalings by 1/h (exact, see dwin) and takes its upwind selections,
// sign tests and tube-test minimum as integer operations on the bit
// patterns.  Same work decomposition as the FP32 kernel: a persistent grid
// of 128-thread CTAs over the active tile list, four x-consecutive points
// per thread, y/z neighbours through shared memory, x through a shuffle,
// face halos from the neighbouring tiles.
#include <cstddef>

#include "ls_internal.cuh"

namespace lsk {

namespace {

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

// ---- FP64 plain step for a power-of-two h, on unscaled differences ----
// With h = 2^-k the oracle's D = d/h is d*2^k exactly, so its squares and
// sums are the unscaled ones times 2^2k, its square root and F*|grad| the
// unscaled ones times 2^k, and dt*(F*|grad|) equals (dt*2^k)*(F*|grad|_u)
// as a real product: the same IEEE results in Eq. 3-5's order without the
// six scalings, as long as every intermediate stays a normal number. The
// windows below guarantee that for |k| <= 16: a nonzero difference within
// [2^-490, 2^490), F zero or within [2^-400, 2^400]. The checks and the
// upwind selections are integer operations on the bit patterns (the
// selected terms are only squared, so the sign of a zero does not matter).
__device__ __forceinline__ bool dwin(double v)
{
    const unsigned hi = (unsigned)__double2hiint(v);
    const unsigned e = (hi >> 20) & 0x7ffu;
    return e - 533u <= 979u || ((hi << 1) | (unsigned)__double2loint(v)) == 0u;
}

__device__ __forceinline__ bool fwin(double v)
{
    const unsigned hi = (unsigned)__double2hiint(v);
    const unsigned e = (hi >> 20) & 0x7ffu;
    return e - 623u <= 800u || ((hi << 1) | (unsigned)__double2loint(v)) == 0u;
}

__device__ __forceinline__ double pos_part(double v) { return __double2hiint(v) >= 0 ? v : 0.0; }
__device__ __forceinline__ double neg_part(double v) { return __double2hiint(v) < 0 ? v : 0.0; }

// Eq. 4 for F > 0 (a = max(D-,0), b = min(D+,0)), Eq. 5 for F < 0
// (a = max(D+,0), b = min(D-,0)), per axis, selected on the bit patterns
__device__ __forceinline__ void sel64u(double F, double& x0, double& x1, double& y0, double& y1,
                                       double& z0, double& z1)
{
    const bool p = __double2hiint(F) >= 0;
    const double ax = p ? x0 : x1, bx = p ? x1 : x0;
    const double ay = p ? y0 : y1, by = p ? y1 : y0;
    const double az = p ? z0 : z1, bz = p ? z1 : z0;
    x0 = pos_part(ax); x1 = neg_part(bx);
    y0 = pos_part(ay); y1 = neg_part(by);
    z0 = pos_part(az); z1 = neg_part(bz);
}

__device__ __forceinline__ bool nonzero(double v)
{
    return (((unsigned)__double2hiint(v) << 1) | (unsigned)__double2loint(v)) != 0u;
}

// both terms of an axis nonzero (a local extremum along it)
__device__ __forceinline__ bool both(double a, double b) { return nonzero(a) && nonzero(b); }

// the rest of Eq. 3 from the sum of squares: F*|grad| with a -0 turned into
// +0 as the oracle's sum with the inactive +0 term does
__device__ __forceinline__ double fin64u(double c, double F, double s, double coef)
{
    double t = __dmul_rn(F, __dsqrt_rn(s));
    if (__double_as_longlong(t) == (long long)0x8000000000000000ull) t = 0.0;
    return __dsub_rn(c, __dmul_rn(coef, t));
}

// per-axis sum of squares, full form RN(RN(a^2) + RN(b^2)), and the short
// form RN(v^2), v the nonzero one of a and b: the same value whenever one
// of them is zero (adding RN(0^2) = +0 to a non-negative number is exact)
__device__ __forceinline__ double ssum_full(double x0, double x1, double y0, double y1, double z0,
                                            double z1)
{
    return __dadd_rn(__dadd_rn(sq_sum(x0, x1), sq_sum(y0, y1)), sq_sum(z0, z1));
}

__device__ __forceinline__ double ssum_short(double x0, double x1, double y0, double y1,
                                             double z0, double z1)
{
    const double vx = nonzero(x0) ? x0 : x1;
    const double vy = nonzero(y0) ? y0 : y1;
    const double vz = nonzero(z0) ? z0 : z1;
    return __dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz));
}

__device__ __forceinline__ D4 ld4(const double* p)
{
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
    D4 r;
    r.v[0] = a.x; r.v[1] = a.y; r.v[2] = b.x; r.v[3] = b.y;
    return r;
}

// ---------------------------------------------------- local scheme, FP64 --
// The oracle's expressions in its order, round-to-nearest intrinsics.
__device__ __forceinline__ double cut64(double a, double beta, double gamma)
{
    if (a <= beta) return 1.0;
    if (a < gamma) {
        const double u = __dsub_rn(a, gamma);
        const double w = __dsub_rn(gamma, beta);
        const double p = __dsub_rn(__dadd_rn(__dmul_rn(2.0, a), gamma), __dmul_rn(3.0, beta));
        return __ddiv_rn(__dmul_rn(__dmul_rn(u, u), p), __dmul_rn(__dmul_rn(w, w), w));
    }
    return 0.0;
}

__device__ __forceinline__ double rei64(double d, double dmx, double dpx, double dmy, double dpy,
                                        double dmz, double dpz, double h, double dtau)
{
    if (d == 0.0) return d;
    double q;
    if (d > 0.0)
        q = __dadd_rn(__dadd_rn(sq_sum(max0(dmx), min0(dpx)), sq_sum(max0(dmy), min0(dpy))),
                      sq_sum(max0(dmz), min0(dpz)));
    else
        q = __dadd_rn(__dadd_rn(sq_sum(max0(dpx), min0(dmx)), sq_sum(max0(dpy), min0(dmy))),
                      sq_sum(max0(dpz), min0(dmz)));
    const double g = __dsqrt_rn(q);
    const double S = __ddiv_rn(d, __dsqrt_rn(__dadd_rn(__dmul_rn(d, d),
                                                         __dmul_rn(__dmul_rn(g, g), __dmul_rn(h, h)))));
    return __dsub_rn(d, __dmul_rn(dtau, __dmul_rn(S, __dsub_rn(g, 1.0))));
}

__device__ __forceinline__ double clamp64(double d, double gamma)
{
    return d < -gamma ? -gamma : (d > gamma ? gamma : d);
}

template <bool FIELD, bool CLASSIFY, int OP = OP_PLAIN>
__global__ void __launch_bounds__(128, 4) k_step_f64(StepArgs a)
{
    __shared__ D4 sm[2][8][8][2];
    __shared__ unsigned long long smin[2];
    __shared__ unsigned nfl[2];   // advance: some point of the tile is in N
    long long prev_k = -1;
    const int tid = threadIdx.x;
    const int xh = tid & 1, ly = (tid >> 1) & 7, lz = tid >> 4;
    const Inst in = a.in;
    const long long n = *a.count;
    if (blockIdx.x == 0 && tid == 0) {
        if (a.updates) atomicAdd(a.updates, (unsigned long long)n * TILE_PTS);
        if (a.updates_timed) atomicAdd(a.updates_timed, (unsigned long long)n * TILE_PTS);
    }
    const double dt = a.sc->dt;
    const double* __restrict__ src = (const double*)a.src;
    double* __restrict__ dst = (double*)a.dst;
    const double* __restrict__ Fp = (const double*)a.F;
    const bool extrap = in.bc == 0;
    const bool pow2h = in.pow2h != 0;
    const double h = in.h, inv_h = in.inv_h;
    // unscaled plain path: h = 2^-k with |k| <= 16 and dt/h exact and normal
    const int kexp = (int)(((unsigned)__double2hiint(inv_h) >> 20) & 0x7ffu) - 1023;
    const int dexp = (int)(((unsigned)__double2hiint(dt) >> 20) & 0x7ffu) - 1023;
    const bool unscaled = OP == OP_PLAIN && pow2h && kexp >= -16 && kexp <= 16 &&
                          dexp >= -900 && dexp <= 900;
    const double coef = __dmul_rn(dt, inv_h);
    const long long sy = (long long)in.tnx * TILE_PTS;
    const long long sz = (long long)in.tnx * in.tny * TILE_PTS;
    const int off = tid * 4;
    int buf = 0;
    int prev_t = -1;
    for (long long k = blockIdx.x; k < n; k += gridDim.x) {
        const int t = __ldg(a.list + k);
        const unsigned info = __ldg(a.info + k);
        const double* tp = src + (size_t)t * TILE_PTS;
        const D4 c = ld4(tp + off);
        D4 f;
        if (FIELD) f = ld4(Fp + (size_t)t * TILE_PTS + off);
        else { f.v[0] = f.v[1] = f.v[2] = f.v[3] = in.Fc; }
        const bool xlo_face = (xh == 0) && !(info & NB_XM);
        const bool xhi_face = (xh == 1) && !(info & NB_XP);
        double xo = 0.0;
        if (xh == 0) {
            if (!xlo_face) xo = __ldg(tp - TILE_PTS + lz * 64 + ly * 8 + 7);
        } else {
            if (!xhi_face) xo = __ldg(tp + TILE_PTS + lz * 64 + ly * 8);
        }
        const bool ylo_face = (ly == 0) && !(info & NB_YM);
        const bool yhi_face = (ly == 7) && !(info & NB_YP);
        D4 yo = c;
        if (ly == 0 && !ylo_face) yo = ld4(tp - sy + lz * 64 + 56 + 4 * xh);
        if (ly == 7 && !yhi_face) yo = ld4(tp + sy + lz * 64 + 4 * xh);
        const bool zlo_face = (lz == 0) && !(info & NB_ZM);
        const bool zhi_face = (lz == 7) && !(info & NB_ZP);
        D4 zo = c;
        if (lz == 0 && !zlo_face) zo = ld4(tp - sz + 448 + ly * 8 + 4 * xh);
        if (lz == 7 && !zhi_face) zo = ld4(tp + sz + ly * 8 + 4 * xh);

        sm[buf][lz][ly][xh] = c;
        if (CLASSIFY && tid == 0) smin[buf] = 0x7ff0000000000000ull;
        if (OP == OP_CUT && tid == 0) nfl[buf] = 0u;
        __syncthreads();
        if (CLASSIFY && tid == 0 && prev_t >= 0)
            a.core[prev_t] = (__longlong_as_double((long long)smin[buf ^ 1]) < in.gamma) ? 1 : 0;
        if (OP == OP_CUT && tid == 0 && prev_k >= 0) a.nflag[prev_k] = (uint8_t)nfl[buf ^ 1];

        const D4 ym = (ly > 0) ? sm[buf][lz][ly - 1][xh] : yo;
        const D4 yp = (ly < 7) ? sm[buf][lz][ly + 1][xh] : yo;
        const D4 zm = (lz > 0) ? sm[buf][lz - 1][ly][xh] : zo;
        const D4 zp = (lz < 7) ? sm[buf][lz + 1][ly][xh] : zo;
        const double part = __shfl_xor_sync(0xffffffffu, xh ? c.v[0] : c.v[3], 1);
        double xn[6];  // x values at x0-1 .. x0+4
        xn[0] = xh ? part : xo;
        xn[1] = c.v[0]; xn[2] = c.v[1]; xn[3] = c.v[2]; xn[4] = c.v[3];
        xn[5] = xh ? xo : part;

        // Eq. 11 bits of the thread's four points (local scheme)
        unsigned nb = 0;
        if constexpr (OP == OP_CUT || OP == OP_CUT_CLAMP) {
            const double g = in.gamma;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                bool inn = fabs(c.v[j]) < g;
                inn |= (j > 0 || !xlo_face) && fabs(xn[j]) < g;
                inn |= (j < 3 || !xhi_face) && fabs(xn[j + 2]) < g;
                inn |= !ylo_face && fabs(ym.v[j]) < g;
                inn |= !yhi_face && fabs(yp.v[j]) < g;
                inn |= !zlo_face && fabs(zm.v[j]) < g;
                inn |= !zhi_face && fabs(zp.v[j]) < g;
                nb |= (inn ? 1u : 0u) << j;
            }
            if constexpr (OP == OP_CUT) {
                uint32_t w = nb << (4 * (tid & 7));
                w |= __shfl_xor_sync(0xffffffffu, w, 1);
                w |= __shfl_xor_sync(0xffffffffu, w, 2);
                w |= __shfl_xor_sync(0xffffffffu, w, 4);
                if ((tid & 7) == 0) a.nmask[(size_t)k * 16 + (tid >> 3)] = w;
                if (__any_sync(0xffffffffu, nb != 0u) && (tid & 31) == 0) nfl[buf] = 1u;
            }
            const unsigned inact = info & NB_ALL & ~(unsigned)__ldg(a.nact + k);
            if (inact && a.breaches) {
                const unsigned tb = (fabs(c.v[0]) < g ? 1u : 0u) | (fabs(c.v[1]) < g ? 2u : 0u) |
                                    (fabs(c.v[2]) < g ? 4u : 0u) | (fabs(c.v[3]) < g ? 8u : 0u);
                const unsigned nt = __popc(tb);
                unsigned bad = 0;
                if (xh == 0 && (tb & 1u) && (inact & NB_XM)) bad += 1;
                if (xh == 1 && (tb & 8u) && (inact & NB_XP)) bad += 1;
                if (ly == 0 && (inact & NB_YM)) bad += nt;
                if (ly == 7 && (inact & NB_YP)) bad += nt;
                if (lz == 0 && (inact & NB_ZM)) bad += nt;
                if (lz == 7 && (inact & NB_ZP)) bad += nt;
                if (bad) atomicAdd(a.breaches, (unsigned long long)bad);
            }
        } else if constexpr (OP == OP_REINIT || OP == OP_REINIT_CLAMP) {
            nb = (__ldg(a.nmask + (size_t)k * 16 + (tid >> 3)) >> (4 * (tid & 7))) & 15u;
        }

        D4 o;
        bool done = false;
        if (OP == OP_PLAIN && unscaled) {
            double u[4][6];
            bool ok = fwin(f.v[0]) && fwin(f.v[1]) && fwin(f.v[2]) && fwin(f.v[3]);
            bool conf = false;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const double cj = c.v[j];
                u[j][0] = __dsub_rn(cj, xn[j]);
                u[j][1] = __dsub_rn(xn[j + 2], cj);
                u[j][2] = __dsub_rn(cj, ym.v[j]);
                u[j][3] = __dsub_rn(yp.v[j], cj);
                u[j][4] = __dsub_rn(cj, zm.v[j]);
                u[j][5] = __dsub_rn(zp.v[j], cj);
                if (j == 0 && xlo_face) u[j][0] = extrap ? u[j][1] : 0.0;
                if (j == 3 && xhi_face) u[j][1] = extrap ? u[j][0] : 0.0;
                if (ylo_face) u[j][2] = extrap ? u[j][3] : 0.0;
                if (yhi_face) u[j][3] = extrap ? u[j][2] : 0.0;
                if (zlo_face) u[j][4] = extrap ? u[j][5] : 0.0;
                if (zhi_face) u[j][5] = extrap ? u[j][4] : 0.0;
                sel64u(f.v[j], u[j][0], u[j][1], u[j][2], u[j][3], u[j][4], u[j][5]);
#pragma unroll
                for (int q = 0; q < 6; ++q) ok = ok && dwin(u[j][q]);
                conf = conf || both(u[j][0], u[j][1]) || both(u[j][2], u[j][3]) ||
                       both(u[j][4], u[j][5]);
            }
            // one form for the whole warp (all its lanes reach this vote)
            const bool full_form = __any_sync(0xffffffffu, conf);
            if (ok) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const double sq = full_form
                        ? ssum_full(u[j][0], u[j][1], u[j][2], u[j][3], u[j][4], u[j][5])
                        : ssum_short(u[j][0], u[j][1], u[j][2], u[j][3], u[j][4], u[j][5]);
                    o.v[j] = fin64u(c.v[j], f.v[j], sq, coef);
                }
                done = true;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (OP == OP_PLAIN && done) continue;
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
            if constexpr (OP == OP_PLAIN) {
                o.v[j] = upd64(cj, f.v[j], dmx, dpx, dmy, dpy, dmz, dpz, dt);
            } else if constexpr (OP == OP_CUT || OP == OP_CUT_CLAMP) {
                const double fe = __dmul_rn(f.v[j], cut64(fabs(cj), a.lp.beta, in.gamma));
                double r = upd64(cj, fe, dmx, dpx, dmy, dpy, dmz, dpz, dt);
                if (OP == OP_CUT_CLAMP && ((nb >> j) & 1u)) r = clamp64(r, in.gamma);
                o.v[j] = r;
            } else {
                double r = rei64(cj, dmx, dpx, dmy, dpy, dmz, dpz, h, a.lp.dtau);
                if (OP == OP_REINIT_CLAMP) r = clamp64(r, in.gamma);
                o.v[j] = ((nb >> j) & 1u) ? r : cj;
            }
        }
        double* dp = dst + (size_t)t * TILE_PTS + off;
        *reinterpret_cast<double2*>(dp) = make_double2(o.v[0], o.v[1]);
        *reinterpret_cast<double2*>(dp + 2) = make_double2(o.v[2], o.v[3]);

        if (CLASSIFY) {
            // min |phi| on the bit patterns: for non-negative doubles the
            // integer order is the numeric order
            const unsigned long long ab = 0x7fffffffffffffffull;
            unsigned long long m =
                min(min((unsigned long long)__double_as_longlong(o.v[0]) & ab,
                        (unsigned long long)__double_as_longlong(o.v[1]) & ab),
                    min((unsigned long long)__double_as_longlong(o.v[2]) & ab,
                        (unsigned long long)__double_as_longlong(o.v[3]) & ab));
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, s));
            if ((tid & 31) == 0) atomicMin(&smin[buf], m);
        }
        buf ^= 1;
        prev_t = t;
        prev_k = k;
    }
    if (CLASSIFY || OP == OP_CUT) {
        __syncthreads();
        if (CLASSIFY && tid == 0 && prev_t >= 0)
            a.core[prev_t] = (__longlong_as_double((long long)smin[buf ^ 1]) < in.gamma) ? 1 : 0;
        if (OP == OP_CUT && tid == 0 && prev_k >= 0) a.nflag[prev_k] = (uint8_t)nfl[buf ^ 1];
    }
}

template <typename K>
int occupancy_grid(K kernel, size_t smem, int threads = 128)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
    if (per < 1) per = 1;
    return sms * per;
}

template <bool FIELD, bool CLS, int OP>
cudaError_t launch64_op(const StepArgs& a, cudaStream_t s)
{
    static int full = 0;
    if (!full) full = occupancy_grid(k_step_f64<FIELD, CLS, OP>, 0);
    int grid = full;
    if (a.max_grid > 0 && grid > a.max_grid) grid = a.max_grid;
    k_step_f64<FIELD, CLS, OP><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_local64(const StepArgs& a, cudaStream_t s)
{
    const bool field = a.F != nullptr;
    const bool cls = a.core != nullptr;
    switch (a.op) {
    case OP_CUT:
        if (cls) return cudaErrorInvalidValue;
        return field ? launch64_op<true, false, OP_CUT>(a, s) : launch64_op<false, false, OP_CUT>(a, s);
    case OP_CUT_CLAMP:
        if (field) return cls ? launch64_op<true, true, OP_CUT_CLAMP>(a, s) : launch64_op<true, false, OP_CUT_CLAMP>(a, s);
        return cls ? launch64_op<false, true, OP_CUT_CLAMP>(a, s) : launch64_op<false, false, OP_CUT_CLAMP>(a, s);
    case OP_REINIT:
        if (cls) return cudaErrorInvalidValue;
        return launch64_op<false, false, OP_REINIT>(a, s);
    case OP_REINIT_CLAMP:
        return cls ? launch64_op<false, true, OP_REINIT_CLAMP>(a, s) : launch64_op<false, false, OP_REINIT_CLAMP>(a, s);
    default:
        return cudaErrorInvalidValue;
    }
}

template <bool FIELD, bool CLS>
cudaError_t launch64(const StepArgs& a, cudaStream_t s)
{
    static int full = 0;
    if (!full) full = occupancy_grid(k_step_f64<FIELD, CLS>, 0);
    int grid = full;
    if (a.max_grid > 0 && grid > a.max_grid) grid = a.max_grid;
    k_step_f64<FIELD, CLS><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step64(const StepArgs& a, cudaStream_t s)
{
    const bool field = a.F != nullptr;
    const bool cls = a.core != nullptr;
    if (a.op != OP_PLAIN) return launch_local64(a, s);
    if (field) return cls ? launch64<true, true>(a, s) : launch64<true, false>(a, s);
    return cls ? launch64<false, true>(a, s) : launch64<false, false>(a, s);
}

}  // namespace lsk
