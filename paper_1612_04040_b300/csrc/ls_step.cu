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
// sign(F).  The FP64 path (bit-identical to the definition) is in
// ls_step64.cu.
//
// Optionally (CLASSIFY) the kernel also evaluates the tube test of Eq. 6 on
// the values it has just written: min |phi^{n+1}| over the tile < gamma in
// FP64.  That saves the rebuild a full re-read of the active tiles.
#include <cstddef>

#include "ls_internal.cuh"
#include "ls_stencil.cuh"

namespace lsk {

namespace {

// ------------------------------------------------------------------ FP32 ----
// Pipelined variant: each thread stages, with cp.async, exactly the values it
// needs for a tile S-1 iterations ahead (its 4 centre values and speeds, its
// x-halo value, and the y/z-halo runs for threads on a tile face) into a
// ring of S shared-memory stages, so the latency of the next tiles' loads
// overlaps the arithmetic of the current one.

// one ring stage; without a speed field the stage has no speed block, so a
// deeper ring fits in the same shared memory
template <bool FIELD>
struct Stage32T {
    float4 v[192];   // [0,128): centre values (element offset 4*tid of the tile);
                     // [128,160): y-halo runs [16*(ly==7) + 2*lz + xh];
                     // [160,192): z-halo runs [16*(lz==7) + 2*ly + xh]
    float4 f[FIELD ? 128 : 1];  // speeds (field speed only)
    float xo[128];   // x-halo value of each thread
    int4 meta;       // tile id, info byte, instance, face neighbours not active
};

// FIELD: speed field (else constant per instance); CLASSIFY: fused tube
// test; BATCHED: list entries belong to different instances (per-entry
// instance id, per-instance dt/h, speed, strides and gamma); S: stages;
// OP: OP_PLAIN (Eq. 3) or a pass of the local scheme (single instance).
template <bool FIELD, bool CLASSIFY, bool BATCHED, int S, int OP = OP_PLAIN>
__global__ void __launch_bounds__(128, 8) k_step_f32(StepArgs a)
{

    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Stage32 = Stage32T<FIELD>;
    Stage32* st = reinterpret_cast<Stage32*>(smem_raw);
    __shared__ unsigned smin[S];
    __shared__ unsigned nfl[OP == OP_CUT ? S : 1];  // advance: some point of the tile is in N
    const int tid = threadIdx.x;
    const int xh = tid & 1, ly = (tid >> 1) & 7, lz = tid >> 4;
    // everything this grid reads may come from the previous grid
    pdl_launch_dependents();
    pdl_wait();
    const int n = *a.count;
    // list position of the k-th entry processed: every other launch walks the
    // list backwards, so it starts on the tiles the previous launch wrote
    // last, which are still in L2
    const bool rev = a.reverse != 0;
    auto ent = [&](int k) { return rev ? n - 1 - k : k; };
    if (blockIdx.x == 0 && tid == 0) {
        if (a.updates) atomicAdd(a.updates, (unsigned long long)n * TILE_PTS);
        if (a.updates_timed) atomicAdd(a.updates_timed, (unsigned long long)n * TILE_PTS);
    }
    const float* __restrict__ src = (const float*)a.src;
    float* __restrict__ dst = (float*)a.dst;
    const float* __restrict__ Fp = (const float*)a.F;
    const int* __restrict__ list = a.list;
    const uint8_t* __restrict__ linfo = a.info;
    const uint16_t* __restrict__ linst = a.list_inst;
    const bool extrap = a.in.bc == 0;
    // single instance: uniform parameters
    const float coef1 = BATCHED ? 0.f : a.sc->coef;
    const float Fc1 = BATCHED ? 0.f : (float)a.in.Fc;
    const double gamma1 = a.in.gamma;
    const int sy1 = a.in.tnx * TILE_PTS;
    const int sz1 = a.in.tnx * a.in.tny * TILE_PTS;
    const int stride = gridDim.x;
    // per-thread halo sources (offsets from the tile start, without the
    // neighbour-tile stride for y/z), the info bit that says the neighbour
    // exists (0 = no halo on that axis) and the smem slots
    const int x_off = xh ? (TILE_PTS + lz * 64 + ly * 8) : (-TILE_PTS + lz * 64 + ly * 8 + 7);
    const unsigned x_bit = xh ? NB_XP : NB_XM;
    const int y_in = (ly == 0) ? (lz * 64 + 56 + 4 * xh) : (lz * 64 + 4 * xh);
    const int y_sgn = (ly == 0) ? -1 : 1;
    const unsigned y_bit = (ly == 0) ? NB_YM : ((ly == 7) ? NB_YP : 0u);
    const int y_slot = 128 + ((ly == 7) ? 16 : 0) + 2 * lz + xh;
    const int z_in = (lz == 0) ? (448 + ly * 8 + 4 * xh) : (ly * 8 + 4 * xh);
    const int z_sgn = (lz == 0) ? -1 : 1;
    const unsigned z_bit = (lz == 0) ? NB_ZM : ((lz == 7) ? NB_ZP : 0u);
    const int z_slot = 160 + ((lz == 7) ? 16 : 0) + 2 * ly + xh;
    const int y_off1 = y_sgn * sy1 + y_in;
    const int z_off1 = z_sgn * sz1 + z_in;
    // smem indices of the four y/z neighbour quads and of the partner value
    const int i_ym = (ly > 0) ? tid - 2 : y_slot;
    const int i_yp = (ly < 7) ? tid + 2 : y_slot;
    const int i_zm = (lz > 0) ? tid - 16 : z_slot;
    const int i_zp = (lz < 7) ? tid + 16 : z_slot;
    const int i_pc = 4 * (tid ^ 1) + (xh ? 3 : 0);

    // shared addresses of this thread's slots in stage 0
    const unsigned sm0 = (unsigned)__cvta_generic_to_shared(st);
    constexpr unsigned SB = (unsigned)sizeof(Stage32);
    const unsigned a_c = sm0 + (unsigned)offsetof(Stage32, v) + 16u * tid;
    const unsigned a_f = sm0 + (unsigned)offsetof(Stage32, f) + 16u * tid;
    const unsigned a_x = sm0 + (unsigned)offsetof(Stage32, xo) + 4u * tid;
    const unsigned a_y = sm0 + (unsigned)offsetof(Stage32, v) + 16u * y_slot;
    const unsigned a_z = sm0 + (unsigned)offsetof(Stage32, v) + 16u * z_slot;
    // N masks of the staged entries (reinitialisation passes)
    __shared__ __align__(16) uint32_t nmk[OP >= OP_REINIT ? S : 1][16];
    const unsigned a_m = (unsigned)__cvta_generic_to_shared(&nmk[0][0]) + 16u * (tid & 3);

    // stage list entry kk = (t, info, instance) into ring slot s
    auto issue = [&](unsigned t, unsigned info, unsigned inst, int s, int kk) {
        const unsigned base = t * TILE_PTS;
        const float* tp = src + base;
        const unsigned so = (unsigned)s * SB;
        Stage32& Sg = st[s];
        if (tid == 0) {
            Sg.meta = make_int4((int)t, (int)info, (int)inst, 0);
            if (CLASSIFY) smin[s] = 0x7f800000u;
            if (OP == OP_CUT) nfl[s] = 0u;
        }
        int y_off = y_off1, z_off = z_off1;
        if (BATCHED) {
            const int tnx = a.insts[inst].tnx, tny = a.insts[inst].tny;
            y_off = y_sgn * (tnx * TILE_PTS) + y_in;
            z_off = z_sgn * (tnx * tny * TILE_PTS) + z_in;
        }
        cp_async16s(a_c + so, tp + 4 * tid);
        if (FIELD) cp_async16s(a_f + so, Fp + base + 4 * tid);
        cp_async4s(a_x + so, tp + x_off, (info & x_bit) != 0);
        cp_async16s(a_y + so, tp + y_off, (info & y_bit) != 0);
        cp_async16s(a_z + so, tp + z_off, (info & z_bit) != 0);
        if (OP >= OP_REINIT && tid < 4)
            cp_async16s(a_m + 64u * (unsigned)s, a.nmask + (size_t)ent(kk) * 16 + 4 * tid);
    };
    // inst: the entry's instance (batched); for the local scheme's advance
    // (single instance) the entry's active face-neighbour bits instead
    auto fetch = [&](int k, unsigned& t, unsigned& info, unsigned& inst) {
        k = ent(k);
        t = (unsigned)__ldg(list + k);
        info = __ldg(linfo + k);
        if (BATCHED) inst = (unsigned)__ldg(linst + k);
        else if (OP == OP_CUT || OP == OP_CUT_CLAMP) inst = __ldg(a.nact + k);
        else inst = 0u;
    };
    auto gamma_of = [&](int inst) -> double { return BATCHED ? a.insts[inst].gamma : gamma1; };

    int kn = blockIdx.x;  // next list entry to stage
#pragma unroll
    for (int s = 0; s < S - 1; ++s) {
        if (kn < n) {
            unsigned t, info, inst;
            fetch(kn, t, info, inst);
            issue(t, info, inst, s, kn);
        }
        cp_async_commit();
        kn += stride;
    }
    // the next two list entries, fetched two iterations ahead of their staging
    unsigned t1 = 0, i1 = 0, n1 = 0, t2 = 0, i2 = 0, n2 = 0;
    if (kn < n) fetch(kn, t1, i1, n1);
    if (kn + stride < n) fetch(kn + stride, t2, i2, n2);
    int cur = 0;
    int prev = -1;
    int prev_t = -1, prev_k = -1, prev_inst = 0;
    for (int k = blockIdx.x; k < n; k += stride) {
        cp_async_wait<S - 2>();
        __syncthreads();
        if (CLASSIFY && tid == 0 && prev >= 0)
            a.core[prev_t] = ((double)__uint_as_float(smin[prev]) < gamma_of(prev_inst)) ? 1 : 0;
        if (OP == OP_CUT && tid == 0 && prev >= 0) a.nflag[prev_k] = (uint8_t)nfl[prev];
        {
            const int sn = cur == 0 ? S - 1 : cur - 1;
            if (kn < n) issue(t1, i1, n1, sn, kn);
            cp_async_commit();
            kn += stride;
            t1 = t2;
            i1 = i2;
            n1 = n2;
            if (kn + stride < n) fetch(kn + stride, t2, i2, n2);
        }
        const Stage32& Sg = st[cur];
        const int t = Sg.meta.x;
        const unsigned info = (unsigned)Sg.meta.y;
        const int inst = Sg.meta.z;
        const float coef = BATCHED ? a.sc[inst].coef : coef1;
        const float Fc = BATCHED ? a.sc[inst].Fc : Fc1;
        const float4 c = Sg.v[tid];
        const float4 f = FIELD ? Sg.f[tid] : make_float4(Fc, Fc, Fc, Fc);
        const float4 ym = Sg.v[i_ym];
        const float4 yp = Sg.v[i_yp];
        const float4 zm = Sg.v[i_zm];
        const float4 zp = Sg.v[i_zp];
        const float pcv = reinterpret_cast<const float*>(Sg.v)[i_pc];
        const float xo = Sg.xo[tid];
        const float xm0 = xh ? pcv : xo;
        const float xp3 = xh ? xo : pcv;

        float4 o;
        if constexpr (OP == OP_PLAIN) {
            if (info == (NB_ALL | SG_POS)) {
                o = upd4<1, false>(c, f, xm0, xp3, ym, yp, zm, zp, coef, extrap, false, false,
                                   false, false, false, false);
            } else if (info == (NB_ALL | SG_NEG)) {
                o = upd4<-1, false>(c, f, xm0, xp3, ym, yp, zm, zp, coef, extrap, false, false,
                                    false, false, false, false);
            } else {
                const bool xlo = (xh == 0) && !(info & NB_XM);
                const bool xhi = (xh == 1) && !(info & NB_XP);
                const bool ylo = (ly == 0) && !(info & NB_YM);
                const bool yhi = (ly == 7) && !(info & NB_YP);
                const bool zlo = (lz == 0) && !(info & NB_ZM);
                const bool zhi = (lz == 7) && !(info & NB_ZP);
                o = upd4<0, true>(c, f, xm0, xp3, ym, yp, zm, zp, coef, extrap, xlo, xhi, ylo,
                                  yhi, zlo, zhi);
            }
        } else {
            const bool xlo = (xh == 0) && !(info & NB_XM);
            const bool xhi = (xh == 1) && !(info & NB_XP);
            const bool ylo = (ly == 0) && !(info & NB_YM);
            const bool yhi = (ly == 7) && !(info & NB_YP);
            const bool zlo = (lz == 0) && !(info & NB_ZM);
            const bool zhi = (lz == 7) && !(info & NB_ZP);
            if constexpr (OP == OP_CUT || OP == OP_CUT_CLAMP) {
                // Eq. 8: the plain update with the speed c(|phi^n|) F (c >= 0
                // keeps the tile's speed-sign class)
                const float4 fs = make_float4(f.x * cut32(fabsf(c.x), a.lp), f.y * cut32(fabsf(c.y), a.lp),
                                              f.z * cut32(fabsf(c.z), a.lp), f.w * cut32(fabsf(c.w), a.lp));
                if (info == (NB_ALL | SG_POS))
                    o = upd4<1, false>(c, fs, xm0, xp3, ym, yp, zm, zp, coef, extrap, false, false,
                                       false, false, false, false);
                else if (info == (NB_ALL | SG_NEG))
                    o = upd4<-1, false>(c, fs, xm0, xp3, ym, yp, zm, zp, coef, extrap, false, false,
                                        false, false, false, false);
                else
                    o = upd4<0, true>(c, fs, xm0, xp3, ym, yp, zm, zp, coef, extrap, xlo, xhi, ylo,
                                      yhi, zlo, zhi);
                const unsigned nb =
                    (info & NB_ALL) == NB_ALL
                        ? n_nibble<false>(c, xm0, xp3, ym, yp, zm, zp, false, false, false, false,
                                          false, false, a.lp.gamma_up)
                        : n_nibble<true>(c, xm0, xp3, ym, yp, zm, zp, xlo, xhi, ylo, yhi, zlo, zhi,
                                         a.lp.gamma_up);
                if constexpr (OP == OP_CUT) {
                    // 16 words of N bits per entry; bit 4*tid + j = point j
                    uint32_t w = nb << (4 * (tid & 7));
                    w |= __shfl_xor_sync(0xffffffffu, w, 1);
                    w |= __shfl_xor_sync(0xffffffffu, w, 2);
                    w |= __shfl_xor_sync(0xffffffffu, w, 4);
                    if ((tid & 7) == 0) a.nmask[(size_t)ent(k) * 16 + (tid >> 3)] = w;
                    if (__any_sync(0xffffffffu, nb != 0u) && (tid & 31) == 0) nfl[cur] = 1u;
                } else {
                    const float gn = a.lp.gamma_up;
                    if (nb & 1u) o.x = fminf(fmaxf(o.x, -gn), gn);
                    if (nb & 2u) o.y = fminf(fmaxf(o.y, -gn), gn);
                    if (nb & 4u) o.z = fminf(fmaxf(o.z, -gn), gn);
                    if (nb & 8u) o.w = fminf(fmaxf(o.w, -gn), gn);
                }
                // face neighbours inside the domain but not active
                const unsigned inact = info & NB_ALL & ~(unsigned)inst;
                if (inact) count_breaches(a, c, inact, xh, ly, lz);
            } else {
                const unsigned nb = (nmk[cur][tid >> 3] >> (4 * (tid & 7))) & 15u;
                constexpr bool CL = OP == OP_REINIT_CLAMP;
                if ((info & NB_ALL) == NB_ALL)
                    o = rei_tile<false, CL>(c, xm0, xp3, ym, yp, zm, zp, nb, a.lp, extrap, false,
                                            false, false, false, false, false);
                else
                    o = rei_tile<true, CL>(c, xm0, xp3, ym, yp, zm, zp, nb, a.lp, extrap, xlo, xhi,
                                           ylo, yhi, zlo, zhi);
            }
        }
        *reinterpret_cast<float4*>(dst + (unsigned)t * TILE_PTS + 4 * tid) = o;

        if (CLASSIFY) {
            const float mn = fminf(fminf(fabsf(o.x), fabsf(o.y)), fminf(fabsf(o.z), fabsf(o.w)));
            const unsigned wm = __reduce_min_sync(0xffffffffu, __float_as_uint(mn));
            if ((tid & 31) == 0) atomicMin(&smin[cur], wm);
        }
        prev = cur;
        prev_t = t;
        prev_k = ent(k);
        prev_inst = inst;
        cur = cur + 1 == S ? 0 : cur + 1;
    }
    if (CLASSIFY || OP == OP_CUT) {
        __syncthreads();
        if (CLASSIFY && tid == 0 && prev >= 0)
            a.core[prev_t] = ((double)__uint_as_float(smin[prev]) < gamma_of(prev_inst)) ? 1 : 0;
        if (OP == OP_CUT && tid == 0 && prev >= 0) a.nflag[prev_k] = (uint8_t)nfl[prev];
    }
    cp_async_wait<0>();
}


// 8 points per thread: 64-thread CTAs, thread (xh, ly, lzp) owns the quads of
// planes lz = 2 lzp and 2 lzp + 1, so each quad's z-neighbour on the other
// plane is already in registers and the per-tile work (staging addresses,
// branching, barrier, store) is spread over twice as many points.  Same
// stage layout, same arithmetic per point (bit-identical results).  OP:
// the plain step, or a reinitialisation pass of the local scheme (Eq. 12 on
// the points of N, whose 512-bit mask per entry is staged with the tile;
// the sign classes are voted per warp and quad set, as in the 4-point pass).
// (the reinitialisation passes: 10 CTAs of up to 102 registers per SM,
// 37.4 us per pass at 512^3 against 40.2 / 41.5 / 44.5 with 12 / 16 / 20
// and 38.5 / 37.9 / 38.3 with 8 / 9 / 11)
template <bool FIELD, bool CLASSIFY, bool BATCHED, int S, int OP = OP_PLAIN>
__global__ void __launch_bounds__(64, OP >= OP_REINIT ? 10 : 16) k_step_f32_z2(StepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Stage32 = Stage32T<FIELD>;
    Stage32* st = reinterpret_cast<Stage32*>(smem_raw);
    __shared__ unsigned smin[S];
    // N masks of the staged entries (reinitialisation passes)
    __shared__ __align__(16) uint32_t nmk[OP >= OP_REINIT ? S : 1][16];
    const int tid = threadIdx.x;
    const int xh = tid & 1, ly = (tid >> 1) & 7, lzp = tid >> 4;
    const int q0 = tid + 16 * lzp, q1 = q0 + 16;
    const int lz0 = 2 * lzp;
    // what this grid reads may come from the previous grid; when that grid
    // was a pass over the same list (early), only the tiles' values and N
    // bits do, so the first entries are loaded before the wait
    pdl_launch_dependents();
    const bool early = a.early != 0;
    if (!early) pdl_wait();
    const int n = *a.count;
    // list position of the k-th entry processed: every other launch walks the
    // list backwards, so it starts on the tiles the previous launch wrote
    // last, which are still in L2
    const bool rev = a.reverse != 0;
    auto ent = [&](int k) { return rev ? n - 1 - k : k; };
    if (blockIdx.x == 0 && tid == 0) {
        if (a.updates) atomicAdd(a.updates, (unsigned long long)n * TILE_PTS);
        if (a.updates_timed) atomicAdd(a.updates_timed, (unsigned long long)n * TILE_PTS);
    }
    const float* __restrict__ src = (const float*)a.src;
    float* __restrict__ dst = (float*)a.dst;
    const float* __restrict__ Fp = (const float*)a.F;
    const int* __restrict__ list = a.list;
    const uint8_t* __restrict__ linfo = a.info;
    const uint16_t* __restrict__ linst = a.list_inst;
    const bool extrap = a.in.bc == 0;
    const float coef1 = BATCHED ? 0.f : a.sc->coef;
    const float Fc1 = BATCHED ? 0.f : (float)a.in.Fc;
    const double gamma1 = a.in.gamma;
    const int sy1 = a.in.tnx * TILE_PTS;
    const int sz1 = a.in.tnx * a.in.tny * TILE_PTS;
    // (rounds spread evenly over the CTAs, as in the one-warp kernel,
    // measured slower here: reinitialisation pass 38.7 against 37.4 us)
    const int stride = gridDim.x;
    const int x_off0 = xh ? (TILE_PTS + lz0 * 64 + ly * 8) : (-TILE_PTS + lz0 * 64 + ly * 8 + 7);
    const unsigned x_bit = xh ? NB_XP : NB_XM;
    const int y_in = (ly == 0) ? (lz0 * 64 + 56 + 4 * xh) : (lz0 * 64 + 4 * xh);
    const int y_sgn = (ly == 0) ? -1 : 1;
    const unsigned y_bit = (ly == 0) ? NB_YM : ((ly == 7) ? NB_YP : 0u);
    const int y_slot0 = 128 + ((ly == 7) ? 16 : 0) + 2 * lz0 + xh;
    const int y_slot1 = y_slot0 + 2;
    const int z_in = (lzp == 0) ? (448 + ly * 8 + 4 * xh) : (ly * 8 + 4 * xh);
    const int z_sgn = (lzp == 0) ? -1 : 1;
    const unsigned z_bit = (lzp == 0) ? NB_ZM : ((lzp == 3) ? NB_ZP : 0u);
    const int z_slot = 160 + ((lzp == 3) ? 16 : 0) + 2 * ly + xh;
    const int y_off1 = y_sgn * sy1 + y_in;
    const int z_off1 = z_sgn * sz1 + z_in;
    const int i_ym0 = (ly > 0) ? q0 - 2 : y_slot0;
    const int i_yp0 = (ly < 7) ? q0 + 2 : y_slot0;
    const int i_ym1 = (ly > 0) ? q1 - 2 : y_slot1;
    const int i_yp1 = (ly < 7) ? q1 + 2 : y_slot1;
    const int i_zm0 = (lzp > 0) ? q0 - 16 : z_slot;
    const int i_zp1 = (lzp < 3) ? q1 + 16 : z_slot;
    const int i_pc0 = 4 * (q0 ^ 1) + (xh ? 3 : 0);
    const int i_pc1 = 4 * (q1 ^ 1) + (xh ? 3 : 0);

    const unsigned sm0 = (unsigned)__cvta_generic_to_shared(st);
    constexpr unsigned SB = (unsigned)sizeof(Stage32);
    const unsigned a_c0 = sm0 + (unsigned)offsetof(Stage32, v) + 16u * q0;
    const unsigned a_f0 = sm0 + (unsigned)offsetof(Stage32, f) + 16u * q0;
    const unsigned a_x0 = sm0 + (unsigned)offsetof(Stage32, xo) + 4u * q0;
    const unsigned a_y0 = sm0 + (unsigned)offsetof(Stage32, v) + 16u * y_slot0;
    const unsigned a_z = sm0 + (unsigned)offsetof(Stage32, v) + 16u * z_slot;
    const unsigned a_m = (unsigned)__cvta_generic_to_shared(&nmk[0][0]) + 16u * (tid & 3);

    auto issue = [&](unsigned t, unsigned info, unsigned inst, int s, int kk) {
        if (OP >= OP_REINIT && tid < 4)
            cp_async16s(a_m + 64u * (unsigned)s, a.nmask + (size_t)ent(kk) * 16 + 4 * tid);
        const unsigned base = t * TILE_PTS;
        const float* tp = src + base;
        const unsigned so = (unsigned)s * SB;
        Stage32& Sg = st[s];
        if (tid == 0) {
            Sg.meta = make_int4((int)t, (int)info, (int)inst, 0);
            if (CLASSIFY) smin[s] = 0x7f800000u;
        }
        int y_off = y_off1, z_off = z_off1;
        if (BATCHED) {
            const int tnx = a.insts[inst].tnx, tny = a.insts[inst].tny;
            y_off = y_sgn * (tnx * TILE_PTS) + y_in;
            z_off = z_sgn * (tnx * tny * TILE_PTS) + z_in;
        }
        cp_async16s(a_c0 + so, tp + 4 * q0);
        cp_async16s(a_c0 + so + 256u, tp + 4 * q1);
        if (FIELD) {
            cp_async16s(a_f0 + so, Fp + base + 4 * q0);
            cp_async16s(a_f0 + so + 256u, Fp + base + 4 * q1);
        }
        const bool px = (info & x_bit) != 0, py = (info & y_bit) != 0;
        cp_async4s(a_x0 + so, tp + x_off0, px);
        cp_async4s(a_x0 + so + 64u, tp + x_off0 + 64, px);
        cp_async16s(a_y0 + so, tp + y_off, py);
        cp_async16s(a_y0 + so + 32u, tp + y_off + 64, py);
        cp_async16s(a_z + so, tp + z_off, (info & z_bit) != 0);
    };
    auto fetch = [&](int k, unsigned& t, unsigned& info, unsigned& inst) {
        k = ent(k);
        t = (unsigned)__ldg(list + k);
        info = __ldg(linfo + k);
        inst = BATCHED ? (unsigned)__ldg(linst + k) : 0u;
    };
    auto gamma_of = [&](int inst) -> double { return BATCHED ? a.insts[inst].gamma : gamma1; };

    int kn = blockIdx.x;
    unsigned pt[S - 1], pi[S - 1], pn[S - 1];
#pragma unroll
    for (int s = 0; s < S - 1; ++s)
        if (kn + s * stride < n) fetch(kn + s * stride, pt[s], pi[s], pn[s]);
    unsigned t1 = 0, i1 = 0, n1 = 0, t2 = 0, i2 = 0, n2 = 0;
    if (kn + (S - 1) * stride < n) fetch(kn + (S - 1) * stride, t1, i1, n1);
    if (kn + S * stride < n) fetch(kn + S * stride, t2, i2, n2);
    if (early) pdl_wait();
#pragma unroll
    for (int s = 0; s < S - 1; ++s) {
        if (kn < n) issue(pt[s], pi[s], pn[s], s, kn);
        cp_async_commit();
        kn += stride;
    }
    int cur = 0, prev = -1, prev_t = -1, prev_inst = 0;
    for (int k = blockIdx.x; k < n; k += stride) {
        cp_async_wait<S - 2>();
        __syncthreads();
        if (CLASSIFY && tid == 0 && prev >= 0)
            a.core[prev_t] = ((double)__uint_as_float(smin[prev]) < gamma_of(prev_inst)) ? 1 : 0;
        {
            const int sn = cur == 0 ? S - 1 : cur - 1;
            if (kn < n) issue(t1, i1, n1, sn, kn);
            cp_async_commit();
            kn += stride;
            t1 = t2;
            i1 = i2;
            n1 = n2;
            if (kn + stride < n) fetch(kn + stride, t2, i2, n2);
        }
        const Stage32& Sg = st[cur];
        const int t = Sg.meta.x;
        const unsigned info = (unsigned)Sg.meta.y;
        const int inst = Sg.meta.z;
        const float coef = BATCHED ? a.sc[inst].coef : coef1;
        const float Fc = BATCHED ? a.sc[inst].Fc : Fc1;
        const float4 c0 = Sg.v[q0], c1 = Sg.v[q1];
        const float4 f0 = FIELD ? Sg.f[q0] : make_float4(Fc, Fc, Fc, Fc);
        const float4 f1 = FIELD ? Sg.f[q1] : make_float4(Fc, Fc, Fc, Fc);
        const float4 ym0 = Sg.v[i_ym0], yp0 = Sg.v[i_yp0];
        const float4 ym1 = Sg.v[i_ym1], yp1 = Sg.v[i_yp1];
        const float4 zm0 = Sg.v[i_zm0], zp1 = Sg.v[i_zp1];
        const float pc0 = reinterpret_cast<const float*>(Sg.v)[i_pc0];
        const float pc1 = reinterpret_cast<const float*>(Sg.v)[i_pc1];
        const float xo0 = Sg.xo[q0], xo1 = Sg.xo[q1];
        const float xm0a = xh ? pc0 : xo0, xp3a = xh ? xo0 : pc0;
        const float xm0b = xh ? pc1 : xo1, xp3b = xh ? xo1 : pc1;
        float4 o0, o1;
        if constexpr (OP >= OP_REINIT) {
            // Eq. 12 on the thread's two quads (points of N only)
            const unsigned nb0 = (nmk[cur][q0 >> 3] >> (4 * (q0 & 7))) & 15u;
            const unsigned nb1 = (nmk[cur][q1 >> 3] >> (4 * (q1 & 7))) & 15u;
            constexpr bool CL = OP == OP_REINIT_CLAMP;
            if ((info & NB_ALL) == NB_ALL) {
                o0 = rei_tile<false, CL>(c0, xm0a, xp3a, ym0, yp0, zm0, c1, nb0, a.lp, extrap, false, false,
                                         false, false, false, false);
                o1 = rei_tile<false, CL>(c1, xm0b, xp3b, ym1, yp1, c0, zp1, nb1, a.lp, extrap, false, false,
                                         false, false, false, false);
            } else {
                const bool xlo = (xh == 0) && !(info & NB_XM);
                const bool xhi = (xh == 1) && !(info & NB_XP);
                const bool ylo = (ly == 0) && !(info & NB_YM);
                const bool yhi = (ly == 7) && !(info & NB_YP);
                const bool zlo = (lzp == 0) && !(info & NB_ZM);
                const bool zhi = (lzp == 3) && !(info & NB_ZP);
                o0 = rei_tile<true, CL>(c0, xm0a, xp3a, ym0, yp0, zm0, c1, nb0, a.lp, extrap, xlo, xhi, ylo,
                                        yhi, zlo, false);
                o1 = rei_tile<true, CL>(c1, xm0b, xp3b, ym1, yp1, c0, zp1, nb1, a.lp, extrap, xlo, xhi, ylo,
                                        yhi, false, zhi);
            }
        } else if (info == (NB_ALL | SG_POS)) {
            o0 = upd4<1, false>(c0, f0, xm0a, xp3a, ym0, yp0, zm0, c1, coef, extrap, false, false, false, false, false, false);
            o1 = upd4<1, false>(c1, f1, xm0b, xp3b, ym1, yp1, c0, zp1, coef, extrap, false, false, false, false, false, false);
        } else if (info == (NB_ALL | SG_NEG)) {
            o0 = upd4<-1, false>(c0, f0, xm0a, xp3a, ym0, yp0, zm0, c1, coef, extrap, false, false, false, false, false, false);
            o1 = upd4<-1, false>(c1, f1, xm0b, xp3b, ym1, yp1, c0, zp1, coef, extrap, false, false, false, false, false, false);
        } else {
            const bool xlo = (xh == 0) && !(info & NB_XM);
            const bool xhi = (xh == 1) && !(info & NB_XP);
            const bool ylo = (ly == 0) && !(info & NB_YM);
            const bool yhi = (ly == 7) && !(info & NB_YP);
            const bool zlo = (lzp == 0) && !(info & NB_ZM);
            const bool zhi = (lzp == 3) && !(info & NB_ZP);
            o0 = upd4<0, true>(c0, f0, xm0a, xp3a, ym0, yp0, zm0, c1, coef, extrap, xlo, xhi, ylo, yhi, zlo, false);
            o1 = upd4<0, true>(c1, f1, xm0b, xp3b, ym1, yp1, c0, zp1, coef, extrap, xlo, xhi, ylo, yhi, false, zhi);
        }
        float* dp = dst + (unsigned)t * TILE_PTS;
        *reinterpret_cast<float4*>(dp + 4 * q0) = o0;
        *reinterpret_cast<float4*>(dp + 4 * q1) = o1;
        if (CLASSIFY) {
            const float mn = fminf(fminf(fminf(fabsf(o0.x), fabsf(o0.y)), fminf(fabsf(o0.z), fabsf(o0.w))),
                                   fminf(fminf(fabsf(o1.x), fabsf(o1.y)), fminf(fabsf(o1.z), fabsf(o1.w))));
            const unsigned wm = __reduce_min_sync(0xffffffffu, __float_as_uint(mn));
            if ((tid & 31) == 0) atomicMin(&smin[cur], wm);
        }
        prev = cur;
        prev_t = t;
        prev_inst = inst;
        cur = cur + 1 == S ? 0 : cur + 1;
    }
    if (CLASSIFY) {
        __syncthreads();
        if (tid == 0 && prev >= 0)
            a.core[prev_t] = ((double)__uint_as_float(smin[prev]) < gamma_of(prev_inst)) ? 1 : 0;
    }
    cp_async_wait<0>();
}

// launch with programmatic stream serialisation (see pdl_wait)
template <typename K>
cudaError_t launch_pdl(K kernel, int grid, int block, size_t smem, const StepArgs& a, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
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

template <bool FIELD, bool CLS, bool BAT, int S>
cudaError_t launch32(const StepArgs& a, int grid_pct, int ppt, cudaStream_t s)
{
    constexpr size_t smem = sizeof(Stage32T<FIELD>) * S;
    static int full4 = 0, full8 = 0;
    int& full = ppt == 8 ? full8 : full4;
    if (!full)
        full = ppt == 8 ? occupancy_grid(k_step_f32_z2<FIELD, CLS, BAT, S>, smem, 64)
                        : occupancy_grid(k_step_f32<FIELD, CLS, BAT, S>, smem, 128);
    int grid = (int)((long long)full * grid_pct / 100);
    if (grid < 1) grid = 1;
    if (a.max_grid > 0 && grid > a.max_grid) grid = a.max_grid;
    if (ppt == 8) return launch_pdl(k_step_f32_z2<FIELD, CLS, BAT, S>, grid, 64, smem, a, s);
    return launch_pdl(k_step_f32<FIELD, CLS, BAT, S>, grid, 128, smem, a, s);
}

template <bool FIELD, bool CLS, bool BAT>
cudaError_t launch32_s(const StepArgs& a, const StepConfig& cfg, cudaStream_t s)
{
    if (cfg.ppt == 16) return launch_step_z4(a, cfg, s);
    switch (cfg.stages) {
    case 2: return launch32<FIELD, CLS, BAT, 2>(a, cfg.grid_pct, cfg.ppt, s);
    case 4: return launch32<FIELD, CLS, BAT, 4>(a, cfg.grid_pct, cfg.ppt, s);
    case 6: return launch32<FIELD, CLS, BAT, 6>(a, cfg.grid_pct, cfg.ppt, s);
    default: return launch32<FIELD, CLS, BAT, 3>(a, cfg.grid_pct, cfg.ppt, s);
    }
}

// local-scheme passes: 4 points per thread; ring depth by stage size
template <bool FIELD, bool CLS, int OP>
cudaError_t launch32_op(const StepArgs& a, int grid_pct, cudaStream_t s)
{
    constexpr int S = FIELD ? 3 : 6;  // the same bytes in flight per CTA
    constexpr size_t smem = sizeof(Stage32T<FIELD>) * S;
    static int full = 0;
    if (!full) full = occupancy_grid(k_step_f32<FIELD, CLS, false, S, OP>, smem, 128);
    int grid = (int)((long long)full * grid_pct / 100);
    if (grid < 1) grid = 1;
    if (a.max_grid > 0 && grid > a.max_grid) grid = a.max_grid;
    return launch_pdl(k_step_f32<FIELD, CLS, false, S, OP>, grid, 128, smem, a, s);
}

// the reinitialisation passes (Eq. 12 on the tiles holding N points): 8
// points per thread, a 2-stage ring (measured with 16 CTAs per SM: 41.4 us
// per pass at 512^3 against 42.8 with 3 stages, 44.4 with 4, 49.0 for the
// 4-point kernel with 6, and 53.5 with one warp per tile; with 10 CTAs per
// SM 37.4 against 37.6 with 3 stages)
template <bool CLS, int OP>
cudaError_t launch_rei_z2(const StepArgs& a, int grid_pct, cudaStream_t s)
{
    constexpr int S = 2;
    constexpr size_t smem = sizeof(Stage32T<false>) * S;
    static int full = 0;
    if (!full) full = occupancy_grid(k_step_f32_z2<false, CLS, false, S, OP>, smem, 64);
    int grid = (int)((long long)full * grid_pct / 100);
    if (grid < 1) grid = 1;
    if (a.max_grid > 0 && grid > a.max_grid) grid = a.max_grid;
    return launch_pdl(k_step_f32_z2<false, CLS, false, S, OP>, grid, 64, smem, a, s);
}

cudaError_t launch_local32(const StepArgs& a, const StepConfig& cfg, cudaStream_t s)
{
    // the advance with one warp per tile when the stencil uses it; the
    // reinitialisation passes with 8 points per thread (launch_rei_z2)
    if (cfg.ppt == 16 && (a.op == OP_CUT || a.op == OP_CUT_CLAMP)) return launch_local_z4(a, cfg, s);
    const bool field = a.F != nullptr;
    const bool cls = a.core != nullptr;
    const int pct = cfg.grid_pct;
    switch (a.op) {
    case OP_CUT:
        if (cls) return cudaErrorInvalidValue;  // the tube test follows the last pass
        return field ? launch32_op<true, false, OP_CUT>(a, pct, s) : launch32_op<false, false, OP_CUT>(a, pct, s);
    case OP_CUT_CLAMP:
        if (field) return cls ? launch32_op<true, true, OP_CUT_CLAMP>(a, pct, s)
                              : launch32_op<true, false, OP_CUT_CLAMP>(a, pct, s);
        return cls ? launch32_op<false, true, OP_CUT_CLAMP>(a, pct, s)
                   : launch32_op<false, false, OP_CUT_CLAMP>(a, pct, s);
    case OP_REINIT:
        if (cls) return cudaErrorInvalidValue;
        return launch_rei_z2<false, OP_REINIT>(a, pct, s);
    case OP_REINIT_CLAMP:
        return cls ? launch_rei_z2<true, OP_REINIT_CLAMP>(a, pct, s)
                   : launch_rei_z2<false, OP_REINIT_CLAMP>(a, pct, s);
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_step(const StepArgs& a, int prec, const StepConfig& cfg, cudaStream_t s)
{
    const bool field = a.F != nullptr;
    const bool cls = a.core != nullptr;
    const bool bat = a.list_inst != nullptr;
    if (a.op != OP_PLAIN) {
        if (bat || !a.nmask) return cudaErrorInvalidValue;  // single-instance contexts only
        return prec == 0 ? launch_local32(a, cfg, s) : launch_step64(a, s);
    }
    if (prec == 0) {
        if (bat) {
            if (field) return cls ? launch32_s<true, true, true>(a, cfg, s) : launch32_s<true, false, true>(a, cfg, s);
            return cls ? launch32_s<false, true, true>(a, cfg, s) : launch32_s<false, false, true>(a, cfg, s);
        }
        if (field) return cls ? launch32_s<true, true, false>(a, cfg, s) : launch32_s<true, false, false>(a, cfg, s);
        return cls ? launch32_s<false, true, false>(a, cfg, s) : launch32_s<false, false, false>(a, cfg, s);
    }
    if (bat) return cudaErrorInvalidValue;  // batched contexts are FP32
    return launch_step64(a, s);
}

}  // namespace lsk
