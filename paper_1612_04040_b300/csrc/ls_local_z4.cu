// ls_local_z4.cu -- the cut-off advance of the local level-set scheme
// (section 1.1, Step 2: Eq. 8 with c of Eq. 7, the N bits of Eq. 11 for the
// reinitialisation passes, the clamp of Eq. 10 when there are none) with one
// warp per 8^3 tile and 16 points per thread, the decomposition of
// ls_step_z4.cu.  The per-point arithmetic is the 4-point pass's
// (ls_stencil.cuh: cut32, upd4, n_nibble, count_breaches) and the N bits keep
// their layout (bit e of the tile's 512-bit mask = element e), so the
// results are the same bits; only the per-tile work is spread over 16
// points.  (The reinitialisation passes take 8 points per thread, the
// 64-thread kernel of ls_step.cu: with one warp per tile they measured
// slower.  The reverse holds for the advance: in that 64-thread kernel,
// at 10, 12 or 16 CTAs per SM, the whole local scheme ran 3-4% slower.)
#include <cstddef>

#include "ls_internal.cuh"
#include "ls_stencil.cuh"

namespace lsk {

namespace {

template <bool FIELD>
struct StageL4 {
    float4 v[192];   // centre quads, y-halo runs, z-halo runs (as the 4-point stage)
    float4 f[FIELD ? 128 : 1];
    float xo[128];
    int4 meta;       // tile id, info byte, active face neighbours
};

template <bool FIELD, bool CLASSIFY, int S, int OP>
__global__ void __launch_bounds__(32, 16) k_local_z4(StepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Stage = StageL4<FIELD>;
    Stage* st = reinterpret_cast<Stage*>(smem_raw);
    const int tid = threadIdx.x;
    const int xh = tid & 1, ly = (tid >> 1) & 7, lzq = tid >> 4;
    const int lz0 = 4 * lzq;
    const int q0 = (tid & 15) + 64 * lzq;
    pdl_launch_dependents();
    pdl_wait();
    const int n = *a.count;
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
    const bool extrap = a.in.bc == 0;
    const float coef = a.sc->coef;
    const float Fc = (float)a.in.Fc;
    const double gamma = a.in.gamma;
    const LocalParams& lp = a.lp;
    const int sy1 = a.in.tnx * TILE_PTS;
    const int sz1 = a.in.tnx * a.in.tny * TILE_PTS;
    const int stride = gridDim.x;
    const int x_off0 = xh ? (TILE_PTS + lz0 * 64 + ly * 8) : (-TILE_PTS + lz0 * 64 + ly * 8 + 7);
    const unsigned x_bit = xh ? NB_XP : NB_XM;
    const int y_in = (ly == 0) ? (lz0 * 64 + 56 + 4 * xh) : (lz0 * 64 + 4 * xh);
    const int y_sgn = (ly == 0) ? -1 : 1;
    const unsigned y_bit = (ly == 0) ? NB_YM : ((ly == 7) ? NB_YP : 0u);
    const int y_slot0 = 128 + ((ly == 7) ? 16 : 0) + 2 * lz0 + xh;
    const int z_in = (lzq == 0) ? (448 + ly * 8 + 4 * xh) : (ly * 8 + 4 * xh);
    const int z_sgn = (lzq == 0) ? -1 : 1;
    const unsigned z_bit = (lzq == 0) ? NB_ZM : NB_ZP;
    const int z_slot = 160 + ((lzq == 1) ? 16 : 0) + 2 * ly + xh;
    const int y_off = y_sgn * sy1 + y_in;
    const int z_off = z_sgn * sz1 + z_in;

    const unsigned sm0 = (unsigned)__cvta_generic_to_shared(st);
    constexpr unsigned SB = (unsigned)sizeof(Stage);
    const unsigned a_c0 = sm0 + (unsigned)offsetof(Stage, v) + 16u * q0;
    const unsigned a_f0 = sm0 + (unsigned)offsetof(Stage, f) + 16u * q0;
    const unsigned a_x0 = sm0 + (unsigned)offsetof(Stage, xo) + 4u * q0;
    const unsigned a_y0 = sm0 + (unsigned)offsetof(Stage, v) + 16u * y_slot0;
    const unsigned a_z = sm0 + (unsigned)offsetof(Stage, v) + 16u * z_slot;

    auto issue = [&](unsigned t, unsigned info, unsigned nact, int s) {
        const unsigned base = t * TILE_PTS;
        const float* tp = src + base;
        const unsigned so = (unsigned)s * SB;
        if (tid == 0) st[s].meta = make_int4((int)t, (int)info, (int)nact, 0);
        const bool px = (info & x_bit) != 0, py = (info & y_bit) != 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            cp_async16s(a_c0 + so + 256u * j, tp + 4 * q0 + 64 * j);
            if (FIELD) cp_async16s(a_f0 + so + 256u * j, Fp + base + 4 * q0 + 64 * j);
            cp_async4s(a_x0 + so + 64u * j, tp + x_off0 + 64 * j, px);
            cp_async16s(a_y0 + so + 32u * j, tp + y_off + 64 * j, py);
        }
        cp_async16s(a_z + so, tp + z_off, (info & z_bit) != 0);
    };
    auto fetch = [&](int k, unsigned& t, unsigned& info, unsigned& nact) {
        k = ent(k);
        t = (unsigned)__ldg(list + k);
        info = __ldg(linfo + k);
        nact = (unsigned)__ldg(a.nact + k);
    };

    int kn = blockIdx.x;
#pragma unroll
    for (int s = 0; s < S - 1; ++s) {
        if (kn < n) {
            unsigned t, info, nact;
            fetch(kn, t, info, nact);
            issue(t, info, nact, s);
        }
        cp_async_commit();
        kn += stride;
    }
    unsigned t1 = 0, i1 = 0, n1 = 0, t2 = 0, i2 = 0, n2 = 0;
    if (kn < n) fetch(kn, t1, i1, n1);
    if (kn + stride < n) fetch(kn + stride, t2, i2, n2);
    int cur = 0;
    for (int k = blockIdx.x; k < n; k += stride) {
        cp_async_wait<S - 2>();
        __syncthreads();
        {
            const int sn = cur == 0 ? S - 1 : cur - 1;
            if (kn < n) issue(t1, i1, n1, sn);
            cp_async_commit();
            kn += stride;
            t1 = t2;
            i1 = i2;
            n1 = n2;
            if (kn + stride < n) fetch(kn + stride, t2, i2, n2);
        }
        const Stage& Sg = st[cur];
        const int t = Sg.meta.x;
        const unsigned info = (unsigned)Sg.meta.y;
        const unsigned nact = (unsigned)Sg.meta.z;
        const bool faces = (info & NB_ALL) != NB_ALL;
        const bool xlo = (xh == 0) && !(info & NB_XM);
        const bool xhi = (xh == 1) && !(info & NB_XP);
        const bool ylo = (ly == 0) && !(info & NB_YM);
        const bool yhi = (ly == 7) && !(info & NB_YP);
        const bool zlo = (lzq == 0) && !(info & NB_ZM);
        const bool zhi = (lzq == 1) && !(info & NB_ZP);
        float4 c[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) c[j] = Sg.v[q0 + 16 * j];
        // neighbours of quad j
        auto nbrs = [&](int j, float4& ym, float4& yp, float4& zm, float4& zp, float& xm0,
                        float& xp3) {
            const int qj = q0 + 16 * j;
            ym = Sg.v[ly > 0 ? qj - 2 : y_slot0 + 2 * j];
            yp = Sg.v[ly < 7 ? qj + 2 : y_slot0 + 2 * j];
            zm = j > 0 ? c[j - 1] : Sg.v[lzq > 0 ? q0 - 16 : z_slot];
            zp = j < 3 ? c[j + 1] : Sg.v[lzq < 1 ? q0 + 64 : z_slot];
            const float pcv = reinterpret_cast<const float*>(Sg.v)[4 * (qj ^ 1) + (xh ? 3 : 0)];
            const float xo = Sg.xo[qj];
            xm0 = xh ? pcv : xo;
            xp3 = xh ? xo : pcv;
        };
        float* dp = dst + (unsigned)t * TILE_PTS;
        float mn = __int_as_float(0x7f800000);
        {
            unsigned anyn = 0u;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int qj = q0 + 16 * j;
                float4 ym, yp, zm, zp;
                float xm0, xp3;
                nbrs(j, ym, yp, zm, zp, xm0, xp3);
                const float4 f = FIELD ? Sg.f[qj] : make_float4(Fc, Fc, Fc, Fc);
                // Eq. 8: the plain update with the speed c(|phi^n|) F
                const float4 fs = make_float4(f.x * cut32(fabsf(c[j].x), lp), f.y * cut32(fabsf(c[j].y), lp),
                                              f.z * cut32(fabsf(c[j].z), lp), f.w * cut32(fabsf(c[j].w), lp));
                const bool zl = zlo && j == 0, zh = zhi && j == 3;
                float4 o;
                if (info == (NB_ALL | SG_POS))
                    o = upd4<1, false>(c[j], fs, xm0, xp3, ym, yp, zm, zp, coef, extrap, false, false,
                                       false, false, false, false);
                else if (info == (NB_ALL | SG_NEG))
                    o = upd4<-1, false>(c[j], fs, xm0, xp3, ym, yp, zm, zp, coef, extrap, false, false,
                                        false, false, false, false);
                else
                    o = upd4<0, true>(c[j], fs, xm0, xp3, ym, yp, zm, zp, coef, extrap, xlo, xhi, ylo,
                                      yhi, zl, zh);
                const unsigned nb =
                    faces ? n_nibble<true>(c[j], xm0, xp3, ym, yp, zm, zp, xlo, xhi, ylo, yhi, zl, zh,
                                           lp.gamma_up)
                          : n_nibble<false>(c[j], xm0, xp3, ym, yp, zm, zp, false, false, false, false,
                                            false, false, lp.gamma_up);
                if constexpr (OP == OP_CUT) {
                    // bits 4 (q & 7) .. +3 of word q >> 3: the eight lanes that
                    // own quads 8w .. 8w + 7 of plane j combine their nibbles
                    uint32_t w = nb << (4 * (qj & 7));
                    w |= __shfl_xor_sync(0xffffffffu, w, 1);
                    w |= __shfl_xor_sync(0xffffffffu, w, 2);
                    w |= __shfl_xor_sync(0xffffffffu, w, 4);
                    if ((tid & 7) == 0) a.nmask[(size_t)ent(k) * 16 + (qj >> 3)] = w;
                    anyn |= nb;
                } else {
                    const float gn = lp.gamma_up;
                    if (nb & 1u) o.x = fminf(fmaxf(o.x, -gn), gn);
                    if (nb & 2u) o.y = fminf(fmaxf(o.y, -gn), gn);
                    if (nb & 4u) o.z = fminf(fmaxf(o.z, -gn), gn);
                    if (nb & 8u) o.w = fminf(fmaxf(o.w, -gn), gn);
                }
                // face neighbours inside the domain but not active
                const unsigned inact = info & NB_ALL & ~nact;
                if (inact) count_breaches(a, c[j], inact, xh, ly, lz0 + j);
                *reinterpret_cast<float4*>(dp + 4 * qj) = o;
                if (CLASSIFY)
                    mn = fminf(mn, fminf(fminf(fabsf(o.x), fabsf(o.y)), fminf(fabsf(o.z), fabsf(o.w))));
            }
            if constexpr (OP == OP_CUT) {
                const bool tile_n = __any_sync(0xffffffffu, anyn != 0u);
                if (tid == 0) a.nflag[ent(k)] = tile_n ? 1u : 0u;
            }
        }
        if (CLASSIFY) {
            const unsigned wm = __reduce_min_sync(0xffffffffu, __float_as_uint(mn));
            if (tid == 0) a.core[t] = ((double)__uint_as_float(wm) < gamma) ? 1 : 0;
        }
        cur = cur + 1 == S ? 0 : cur + 1;
    }
    cp_async_wait<0>();
}

template <typename K>
int occupancy_grid_l4(K kernel, size_t smem)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 32, smem);
    if (per < 1) per = 1;
    return sms * per;
}

template <bool FIELD, bool CLS, int OP>
cudaError_t launch_l4(const StepArgs& a, int grid_pct, cudaStream_t s)
{
    constexpr int S = 2;
    constexpr size_t smem = sizeof(StageL4<FIELD>) * S;
    static int full = 0;
    if (!full) full = occupancy_grid_l4(k_local_z4<FIELD, CLS, S, OP>, smem);
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
    return cudaLaunchKernelEx(&cfg, k_local_z4<FIELD, CLS, S, OP>, a);
}

}  // namespace

cudaError_t launch_local_z4(const StepArgs& a, const StepConfig& cfg, cudaStream_t s)
{
    const bool field = a.F != nullptr;
    const bool cls = a.core != nullptr;
    const int pct = cfg.grid_pct;
    switch (a.op) {
    case OP_CUT:
        if (cls) return cudaErrorInvalidValue;  // the tube test follows the last pass
        return field ? launch_l4<true, false, OP_CUT>(a, pct, s) : launch_l4<false, false, OP_CUT>(a, pct, s);
    case OP_CUT_CLAMP:
        if (field) return cls ? launch_l4<true, true, OP_CUT_CLAMP>(a, pct, s)
                              : launch_l4<true, false, OP_CUT_CLAMP>(a, pct, s);
        return cls ? launch_l4<false, true, OP_CUT_CLAMP>(a, pct, s)
                   : launch_l4<false, false, OP_CUT_CLAMP>(a, pct, s);
    default:
        return cudaErrorInvalidValue;  // the reinitialisation passes: 4 points per thread
    }
}

}  // namespace lsk
