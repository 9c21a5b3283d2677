// ls_step_z4.cu -- the upwind step (Eq. 3-5) with one warp per 8^3 tile and
// 16 points per thread.
//
// Thread (xh, ly, lzq) of the warp owns the four z-adjacent quads of planes
// lz = 4 lzq .. 4 lzq + 3 at (ly, 4 xh .. 4 xh + 3), so three of each
// quad's z neighbours are in its own registers, and the per-tile work
// (list entry, staging addresses, branch on the tile's class, barrier) is
// spread over 16 points instead of 4 (ls_step.cu) or 8.  The tube-test
// minimum of a tile is one warp reduction (no shared-memory atomics).  The
// 4-point kernel's stage layout without its speed block, the same per-point
// arithmetic (ls_stencil.cuh), so the results are the same bits for every
// choice of points per thread.
//
// Staging: the tile's 2 KiB block and its two z faces (256-byte runs) are
// bulk asynchronous copies issued by one lane and completing on the stage's
// mbarrier; the x-halo words and the 32-byte y-halo runs are per-lane
// cp.async as in the other kernels.  The bulk copies do not pass through the
// L1 data cache, which the cp.async requests in flight otherwise share with
// the halo gathers (measured: batch of 256 grids 163.7 -> 157.1 us per
// launch, 512^3 sphere union 60.9 -> 59.8 us).  Small requests do not pay on
// the copy engine: the y runs as sixteen 32-byte bulk copies measured 184 us,
// the x faces as tensor boxes of the neighbours' boundary quads (64 rows of
// 16 bytes) 190 us.
#include <cstddef>

#include "ls_internal.cuh"
#include "ls_stencil.cuh"

namespace lsk {

namespace {

// one ring stage (the layout of the 4-point kernel's stage, without the
// speed block: each thread reads its own 16 speeds straight into registers
// when it computes the tile -- they are nobody's neighbours -- which keeps
// the stage at 3.6 KB and measured 5 % faster than staging them).  The x-halo
// words of planes 4..7 are stored with planes 4 <-> 5 and 6 <-> 7 swapped, so
// that the two half-warps read different banks.  (A y-halo layout free of
// bank conflicts, eight-quad rows with each quarter-warp's halo quads in the
// bank groups its in-tile quads leave free, measured no faster: the 512 bytes
// it adds per stage come out of the L1 capacity the halo gathers use.)
struct StageZ4 {
    float4 v[192];   // [0,128): centre quads; [128,160): y-halo runs [16*(ly==7) + 2*lz + xh];
                     // [160,192): z-halo runs [16*(lz==7) + 2*ly + xh]
    float xo[128];   // x-halo value of each quad, quad q0 + 16 j at q0 + 16 (j ^ lzq)
    int4 meta;       // tile id, info byte, instance
    float2 mf;       // batched: the instance's dt / h and constant speed
    unsigned long long bar;  // completion of the stage's bulk copies
};

// a list entry with what its staging and its update need (batched: the
// instance's tile-row strides, dt / h and speed).  The entry itself is
// loaded three tiles ahead of its staging and, batched, its instance's data
// one tile later, once the instance id has arrived: no load waits on
// another load in the same iteration.
struct EntZ4 {
    unsigned t, info, inst;
    int tnx, tny;
    float coef, Fc;
};

// the four quads of one thread, one class of tile (SGN, FACES as upd4)
template <int SGN, bool FACES, bool FIELD, bool CLASSIFY>
__device__ __forceinline__ void quads4(const StageZ4& Sg, const float4 (&c)[4],
                                       const float4 (&fr)[4], float Fc, float coef, bool extrap,
                                       int q0, int xh, int ly, int lzq,
                                       int y_slot0, int z_slot, bool xlo, bool xhi, bool ylo,
                                       bool yhi, bool zlo, bool zhi, float* dp, float& mn)
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int qj = q0 + 16 * j;
        const float4 f = FIELD ? fr[j] : make_float4(Fc, Fc, Fc, Fc);
        const float4 ym = Sg.v[ly > 0 ? qj - 2 : y_slot0 + 2 * j];
        const float4 yp = Sg.v[ly < 7 ? qj + 2 : y_slot0 + 2 * j];
        const float4 zm = j > 0 ? c[j - 1] : Sg.v[lzq > 0 ? q0 - 16 : z_slot];
        const float4 zp = j < 3 ? c[j + 1] : Sg.v[lzq < 1 ? q0 + 64 : z_slot];
        // the in-tile x neighbour across the quad boundary is in the partner
        // lane's registers (same row, other half)
        const float pcv = __shfl_xor_sync(0xffffffffu, xh ? c[j].x : c[j].w, 1);
        const float xo = Sg.xo[q0 + 16 * (j ^ lzq)];
        const float xm0 = xh ? pcv : xo, xp3 = xh ? xo : pcv;
        const float4 o = upd4<SGN, FACES>(c[j], f, xm0, xp3, ym, yp, zm, zp, coef, extrap, xlo, xhi,
                                          ylo, yhi, zlo && j == 0, zhi && j == 3);
        *reinterpret_cast<float4*>(dp + 4 * qj) = o;
        if (CLASSIFY)
            mn = fminf(mn, fminf(fminf(fabsf(o.x), fabsf(o.y)), fminf(fabsf(o.z), fabsf(o.w))));
    }
}

// FIELD: speed field (else constant per instance); CLASSIFY: fused tube test
// (Eq. 6); BATCHED: per-entry instance; S: ring stages.  16 warps of up to
// 128 registers per SM.  (Without a speed field the kernel also fits in 96
// registers, 21 warps per SM: faster in a short burst, batch of 256 grids
// 163.3 against 166.6 us per launch, but slower sustained under the power
// cap, 177.1 against 172.5 us, and 2 % fewer updates per second over the
// whole run; with a speed field slower either way, 512^3 sphere union 63.4
// against 59.7 us.)
template <bool FIELD, bool CLASSIFY, bool BATCHED, int S>
__global__ void __launch_bounds__(32, 16) k_step_f32_z4(StepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Stage = StageZ4;
    Stage* st = reinterpret_cast<Stage*>(smem_raw);
    const int tid = threadIdx.x;
    const int xh = tid & 1, ly = (tid >> 1) & 7, lzq = tid >> 4;
    const int lz0 = 4 * lzq;
    const int q0 = (tid & 15) + 64 * lzq;  // quad of plane lz0; plane lz0 + j: q0 + 16 j
    // what this grid reads may come from the previous grid; when that grid
    // was a step over the same list (early), only the tiles' values do, so
    // the list entries of the first tiles are loaded before the wait
    pdl_launch_dependents();
    const bool early = a.early != 0;
    if (!early) pdl_wait();
    const int n = *a.count;
    // every other launch walks the list backwards (L2 reuse across launches)
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
    // as many rounds over the list as the whole grid needs, spread evenly
    // over the CTAs (no last round with a fraction of them busy: 512^3
    // sphere union 475.1 -> 476.0 GLUPS)
    const int rounds = (n + (int)gridDim.x - 1) / (int)gridDim.x;
    const int stride = rounds > 0 ? (n + rounds - 1) / rounds : (int)gridDim.x;
    if ((int)blockIdx.x >= stride) return;
    // halo sources of plane lz0 (plane lz0 + j: + 64 j elements)
    const int x_off0 = xh ? (TILE_PTS + lz0 * 64 + ly * 8) : (-TILE_PTS + lz0 * 64 + ly * 8 + 7);
    const unsigned x_bit = xh ? NB_XP : NB_XM;
    const int y_in = (ly == 0) ? (lz0 * 64 + 56 + 4 * xh) : (lz0 * 64 + 4 * xh);
    const int y_sgn = (ly == 0) ? -1 : 1;
    const unsigned y_bit = (ly == 0) ? NB_YM : ((ly == 7) ? NB_YP : 0u);
    const int y_slot0 = 128 + ((ly == 7) ? 16 : 0) + 2 * lz0 + xh;
    // the z-halo quad of the lower half-warp's plane 0 (-z face) and of the
    // upper half-warp's plane 7 (+z face)
    const int z_slot = 160 + ((lzq == 1) ? 16 : 0) + 2 * ly + xh;
    const int y_off1 = y_sgn * sy1 + y_in;
    // a frozen x neighbour's face from its copy (single grid): value
    // (lz0 + j, ly) of this thread's side at xf_off0 + 8 j; faces with their
    // fill bit are read in place by a filling launch, which writes the copy
    float* __restrict__ xf = BATCHED ? nullptr : a.xface;
    const bool xfill = a.xface_fill != 0;
    const int xf_off0 = xh * 64 + lz0 * 8 + ly;
    const unsigned fill_bit = x_bit << 6;  // NACT_FILL_XM / _XP

    const unsigned sm0 = (unsigned)__cvta_generic_to_shared(st);
    constexpr unsigned SB = (unsigned)sizeof(Stage);
    const unsigned a_x0 = sm0 + (unsigned)offsetof(Stage, xo) + 4u * q0;
    const unsigned a_y0 = sm0 + (unsigned)offsetof(Stage, v) + 16u * y_slot0;
    const unsigned a_v = sm0 + (unsigned)offsetof(Stage, v);
    const unsigned a_bar = sm0 + (unsigned)offsetof(Stage, bar);
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s) bulk_mbar_init(a_bar + (unsigned)s * SB);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    unsigned phase = 0u;  // parity of each stage's next completion (bit s)

    auto issue = [&](const EntZ4& e, int s) {
        const unsigned t = e.t, info = e.info, inst = e.inst;
        const unsigned base = t * TILE_PTS;
        const float* tp = src + base;
        const unsigned so = (unsigned)s * SB;
        int y_off = y_off1;
        if (BATCHED) y_off = y_sgn * (e.tnx * TILE_PTS) + y_in;
        if (tid == 0) {
            st[s].meta = make_int4((int)t, (int)info, (int)inst, 0);
            if (BATCHED) st[s].mf = make_float2(e.coef, e.Fc);
            const bool zm = (info & NB_ZM) != 0, zp = (info & NB_ZP) != 0;
            const int sz = BATCHED ? e.tnx * e.tny * TILE_PTS : sz1;
            const unsigned bar = a_bar + so;
            // this stage was last read by generic loads (ordered before by
            // the ring barrier); the bulk copies write it
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bulk_expect_tx(bar, 2048u + (zm ? 256u : 0u) + (zp ? 256u : 0u));
            bulk_g2s(a_v + so, tp, 2048u, bar);
            if (zm) bulk_g2s(a_v + so + 16u * 160u, tp - sz + 448, 256u, bar);  // plane 7 below
            if (zp) bulk_g2s(a_v + so + 16u * 176u, tp + sz, 256u, bar);        // plane 0 above
        }
        const bool px = (info & x_bit) != 0, py = (info & y_bit) != 0;
        // inst: the entry's active face-neighbour and fill bits when xf is set
        const bool fz = !BATCHED && xf && (info & ~inst & x_bit) != 0 && !(xfill && (inst & fill_bit));
        const float* xs = fz ? xf + (size_t)t * XFACE_FLOATS + xf_off0 : tp + x_off0;
        const int xstep = fz ? 8 : 64;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            cp_async4s(a_x0 + so + 64u * (unsigned)(j ^ lzq), xs + xstep * j, px);
            cp_async16s(a_y0 + so + 32u * j, tp + y_off + 64 * j, py);
        }
    };
    auto fetch_entry = [&](int k, EntZ4& e) {
        k = ent(k);
        e.t = (unsigned)__ldg(list + k);
        e.info = __ldg(linfo + k);
        e.inst = BATCHED ? (unsigned)__ldg(linst + k) : (xf ? (unsigned)__ldg(a.nact + k) : 0u);
    };
    auto fetch_inst = [&](EntZ4& e) {
        if (BATCHED) {
            e.tnx = a.insts[e.inst].tnx;
            e.tny = a.insts[e.inst].tny;
            e.coef = a.sc[e.inst].coef;
            e.Fc = a.sc[e.inst].Fc;
        }
    };
    auto fetch = [&](int k, EntZ4& e) {
        fetch_entry(k, e);
        fetch_inst(e);
    };

    // tile ids of the staged entries in the order they are computed, so
    // that a tile's speeds can be requested before the ring wait
    unsigned tq[S - 1];
    EntZ4 e0[S - 1];
    EntZ4 e1_init = {};
    int kn = blockIdx.x;
#pragma unroll
    for (int s = 0; s < S - 1; ++s) {
        tq[s] = 0u;
        if (kn + s * stride < n) {
            fetch(kn + s * stride, e0[s]);
            tq[s] = e0[s].t;
        }
    }
    {
        const int k1 = kn + (S - 1) * stride;
        if (k1 < n) fetch(k1, e1_init);
    }
    if (early) pdl_wait();
#pragma unroll
    for (int s = 0; s < S - 1; ++s) {
        if (kn < n) issue(e0[s], s);
        cp_async_commit();
        kn += stride;
    }
    EntZ4 e1 = e1_init, e2 = {}, e3 = {};
    if (kn + stride < n) fetch(kn + stride, e2);
    if (BATCHED && kn + 2 * stride < n) fetch_entry(kn + 2 * stride, e3);
    int cur = 0;
    for (int k = blockIdx.x; k < n; k += stride) {
        // this tile's speeds (each thread its own 16: nobody's neighbours),
        // requested before the ring wait so that their latency overlaps it
        float4 fr[4];
        if (FIELD) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                fr[j] = __ldg(reinterpret_cast<const float4*>(Fp + (size_t)tq[0] * TILE_PTS + 4 * q0 + 64 * j));
        }
        cp_async_wait<S - 2>();
        {
            const unsigned par = (phase >> cur) & 1u;
            const bool ok = bulk_wait(a_bar + (unsigned)cur * SB, par, 1ll << 26);
            if (!__all_sync(0xffffffffu, ok ? 1 : 0)) {
                // give up: record it, let the copies still in flight land
                // (bounded waits), and leave
                if (tid == 0) {
                    if (a.status) atomicOr(a.status, ST_TIMEOUT);
                    bulk_wait(a_bar + (unsigned)cur * SB, par, 1ll << 20);
                    for (int i = 1; i < S - 1; ++i) {
                        const int s2 = (cur + i) % S;
                        if (k + i * stride < n) bulk_wait(a_bar + (unsigned)s2 * SB, (phase >> s2) & 1u, 1ll << 20);
                    }
                }
                cp_async_wait<0>();
                return;
            }
            phase ^= 1u << cur;
        }
        __syncthreads();
        {
            const int sn = cur == 0 ? S - 1 : cur - 1;
            if (kn < n) issue(e1, sn);
            cp_async_commit();
#pragma unroll
            for (int i = 0; i + 1 < S - 1; ++i) tq[i] = tq[i + 1];
            tq[S - 2] = e1.t;
            kn += stride;
            e1 = e2;
            if (BATCHED) {
                e2 = e3;
                if (kn + stride < n) fetch_inst(e2);
                if (kn + 2 * stride < n) fetch_entry(kn + 2 * stride, e3);
            } else if (kn + stride < n) {
                fetch(kn + stride, e2);
            }
        }
        const Stage& Sg = st[cur];
        const int t = Sg.meta.x;
        const unsigned info = (unsigned)Sg.meta.y;
        const int inst = Sg.meta.z;
        const float coef = BATCHED ? Sg.mf.x : coef1;
        const float Fc = BATCHED ? Sg.mf.y : Fc1;
        // the tube test's gamma, requested before the update hides its latency
        const double g = (CLASSIFY && BATCHED && tid == 0) ? a.insts[inst].gamma : gamma1;
        float4 c[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) c[j] = Sg.v[q0 + 16 * j];
        float* dp = dst + (unsigned)t * TILE_PTS;
        if (!BATCHED && xfill && ((unsigned)inst & fill_bit)) {
#pragma unroll
            for (int j = 0; j < 4; ++j) xf[(size_t)t * XFACE_FLOATS + xf_off0 + 8 * j] = Sg.xo[q0 + 16 * (j ^ lzq)];
        }
        float mn = __int_as_float(0x7f800000);
        if (info == (NB_ALL | SG_POS)) {
            quads4<1, false, FIELD, CLASSIFY>(Sg, c, fr, Fc, coef, extrap, q0, xh, ly, lzq, y_slot0, z_slot,
                                              false, false, false, false, false, false, dp, mn);
        } else if (info == (NB_ALL | SG_NEG)) {
            quads4<-1, false, FIELD, CLASSIFY>(Sg, c, fr, Fc, coef, extrap, q0, xh, ly, lzq, y_slot0, z_slot,
                                               false, false, false, false, false, false, dp, mn);
        } else {
            const bool xlo = (xh == 0) && !(info & NB_XM);
            const bool xhi = (xh == 1) && !(info & NB_XP);
            const bool ylo = (ly == 0) && !(info & NB_YM);
            const bool yhi = (ly == 7) && !(info & NB_YP);
            const bool zlo = (lzq == 0) && !(info & NB_ZM);
            const bool zhi = (lzq == 1) && !(info & NB_ZP);
            quads4<0, true, FIELD, CLASSIFY>(Sg, c, fr, Fc, coef, extrap, q0, xh, ly, lzq, y_slot0, z_slot,
                                             xlo, xhi, ylo, yhi, zlo, zhi, dp, mn);
        }
        if (CLASSIFY) {
            // the warp holds the whole tile: its minimum is the tile's
            const unsigned wm = __reduce_min_sync(0xffffffffu, __float_as_uint(mn));
            if (tid == 0) a.core[t] = ((double)__uint_as_float(wm) < g) ? 1 : 0;
        }
        cur = cur + 1 == S ? 0 : cur + 1;
    }
    cp_async_wait<0>();
}

template <typename K>
int occupancy_grid_z4(K kernel, size_t smem)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 32, smem);
    if (per < 1) per = 1;
    return sms * per;
}

template <bool FIELD, bool CLS, bool BAT, int S>
cudaError_t launch_z4(const StepArgs& a, int grid_pct, cudaStream_t s)
{
    constexpr size_t smem = sizeof(StageZ4) * S;
    static int full = 0;
    if (!full) full = occupancy_grid_z4(k_step_f32_z4<FIELD, CLS, BAT, S>, smem);
    int grid = (int)((long long)full * grid_pct / 100);
    if (grid < 1) grid = 1;
    if (a.max_grid > 0 && grid > a.max_grid) grid = a.max_grid;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(32u);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_step_f32_z4<FIELD, CLS, BAT, S>, a);
}

template <bool FIELD, bool CLS, bool BAT>
cudaError_t launch_z4_s(const StepArgs& a, const StepConfig& cfg, cudaStream_t s)
{
    switch (cfg.stages) {
    case 2: return launch_z4<FIELD, CLS, BAT, 2>(a, cfg.grid_pct, s);
    case 4: return launch_z4<FIELD, CLS, BAT, 4>(a, cfg.grid_pct, s);
    case 6: return launch_z4<FIELD, CLS, BAT, 6>(a, cfg.grid_pct, s);
    default: return launch_z4<FIELD, CLS, BAT, 3>(a, cfg.grid_pct, s);
    }
}

}  // namespace

cudaError_t launch_step_z4(const StepArgs& a, const StepConfig& cfg, cudaStream_t s)
{
    const bool field = a.F != nullptr;
    const bool cls = a.core != nullptr;
    const bool bat = a.list_inst != nullptr;
    if (bat) {
        if (field) return cls ? launch_z4_s<true, true, true>(a, cfg, s) : launch_z4_s<true, false, true>(a, cfg, s);
        return cls ? launch_z4_s<false, true, true>(a, cfg, s) : launch_z4_s<false, false, true>(a, cfg, s);
    }
    if (field) return cls ? launch_z4_s<true, true, false>(a, cfg, s) : launch_z4_s<true, false, false>(a, cfg, s);
    return cls ? launch_z4_s<false, true, false>(a, cfg, s) : launch_z4_s<false, false, false>(a, cfg, s);
}

}  // namespace lsk
