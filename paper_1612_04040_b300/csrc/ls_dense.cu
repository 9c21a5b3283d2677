// ls_dense.cu -- the upwind step (Eq. 3-5) over the whole domain
// (full-domain mode, FP32, single grid): tile columns streamed along z.
//
// The list kernel walks tiles in ascending id order, so a tile's z
// neighbours are a whole xy-plane of tiles apart; on a full 1024^3 domain
// (one plane of tiles is ~100 MB of traffic) they have left L2 by the time
// they are needed.  Here CTA b walks the tile columns col = b, b + G, ...
// and each column along z: the z halos of a tile are the previous and the
// next tile of the same column, which the CTA stages anyway (the ring keeps
// the previous stage and has the next one landed), so no z halo is read
// twice.  x / y halos come from the neighbouring columns, which neighbouring
// CTAs stream at about the same z.  Same per-point arithmetic as the other
// stencils (bit-identical results).
#include <cstddef>

#include "ls_internal.cuh"
#include "ls_stencil.cuh"

namespace lsk {

namespace {

template <bool FIELD>
struct DStage {
    float4 v[160];              // [0,128): centre quads; [128,160): y-halo runs
                                // [16*(ly==7) + 2*lz + xh]
    float4 f[FIELD ? 128 : 1];  // speeds (field speed only)
    float xo[128];              // x-halo value of each thread
    int4 meta;                  // tile id, info byte
};

constexpr int DS = 5;  // ring: previous, current, next (landed), two in flight

template <bool FIELD>
__global__ void __launch_bounds__(128, 8) k_dense_f32(StepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Stage = DStage<FIELD>;
    Stage* st = reinterpret_cast<Stage*>(smem_raw);
    const int tid = threadIdx.x;
    const int xh = tid & 1, ly = (tid >> 1) & 7, lz = tid >> 4;
    pdl_launch_dependents();
    pdl_wait();
    const Inst in = a.in;
    const int tnx = in.tnx, tny = in.tny, tnz = in.tnz;
    const int ncol = tnx * tny;
    const int G = gridDim.x;
    const int mycols = (int)blockIdx.x < ncol ? (ncol - (int)blockIdx.x + G - 1) / G : 0;
    const long long total = (long long)mycols * tnz;
    if (blockIdx.x == 0 && tid == 0) {
        if (a.updates) atomicAdd(a.updates, (unsigned long long)ncol * tnz * TILE_PTS);
        if (a.updates_timed) atomicAdd(a.updates_timed, (unsigned long long)ncol * tnz * TILE_PTS);
    }
    const float* __restrict__ src = (const float*)a.src;
    float* __restrict__ dst = (float*)a.dst;
    const float* __restrict__ Fp = (const float*)a.F;
    const bool extrap = in.bc == 0;
    const float coef = a.sc->coef;
    const float Fc = (float)in.Fc;
    const unsigned const_sgn = in.Fc >= 0.0 ? SG_POS : SG_NEG;
    const int sy = tnx * TILE_PTS;
    // per-thread halo sources and slots (as in the list kernel)
    const int x_off = xh ? (TILE_PTS + lz * 64 + ly * 8) : (-TILE_PTS + lz * 64 + ly * 8 + 7);
    const unsigned x_bit = xh ? NB_XP : NB_XM;
    const int y_in = (ly == 0) ? (lz * 64 + 56 + 4 * xh) : (lz * 64 + 4 * xh);
    const int y_off = ((ly == 0) ? -sy : sy) + y_in;
    const unsigned y_bit = (ly == 0) ? NB_YM : ((ly == 7) ? NB_YP : 0u);
    const int y_slot = 128 + ((ly == 7) ? 16 : 0) + 2 * lz + xh;
    const int i_ym = (ly > 0) ? tid - 2 : y_slot;
    const int i_yp = (ly < 7) ? tid + 2 : y_slot;
    const int i_pc = 4 * (tid ^ 1) + (xh ? 3 : 0);
    const unsigned sm0 = (unsigned)__cvta_generic_to_shared(st);
    constexpr unsigned SB = (unsigned)sizeof(Stage);
    const unsigned a_c = sm0 + (unsigned)offsetof(Stage, v) + 16u * tid;
    const unsigned a_f = sm0 + (unsigned)offsetof(Stage, f) + 16u * tid;
    const unsigned a_x = sm0 + (unsigned)offsetof(Stage, xo) + 4u * tid;
    const unsigned a_y = sm0 + (unsigned)offsetof(Stage, v) + 16u * y_slot;

    // entries are prepared in order (the q-th tile of this CTA: column
    // q / tnz, z index q % tnz), one iteration before they are staged, with a
    // running cursor (no divisions on the way) so that the sign-class load
    // is off the path
    struct Next {
        long long t;
        unsigned info;
        int tz;
    };
    int pci = 0, ptz = 0, pcol = (int)blockIdx.x;
    int pty = pcol / tnx, ptx = pcol - pty * tnx;
    auto prepare = [&]() {
        Next nx{0, 0u, 0};
        if (pci < mycols) {
            nx.t = (long long)ptz * ncol + pcol;
            nx.tz = ptz;
            unsigned nb = 0;
            if (ptx > 0) nb |= NB_XM;
            if (ptx < tnx - 1) nb |= NB_XP;
            if (pty > 0) nb |= NB_YM;
            if (pty < tny - 1) nb |= NB_YP;
            if (ptz > 0) nb |= NB_ZM;
            if (ptz < tnz - 1) nb |= NB_ZP;
            nx.info = nb | (a.tile_sgn ? (unsigned)__ldg(a.tile_sgn + nx.t) : const_sgn);
            if (++ptz == tnz) {
                ptz = 0;
                ++pci;
                pcol += G;
                pty = pcol / tnx;
                ptx = pcol - pty * tnx;
            }
        }
        return nx;
    };
    auto issue = [&](long long q, const Next& nx) {
        if (q < total) {
            const int tz = nx.tz;
            const unsigned info = nx.info;
            const long long t = nx.t;
            const int s = (int)(q % DS);
            const unsigned so = (unsigned)s * SB;
            const float* tp = src + t * TILE_PTS;
            if (tid == 0) st[s].meta = make_int4((int)t, (int)info, tz, 0);
            cp_async16s(a_c + so, tp + 4 * tid);
            if (FIELD) cp_async16s(a_f + so, Fp + t * TILE_PTS + 4 * tid);
            cp_async4s(a_x + so, tp + x_off, (info & x_bit) != 0);
            cp_async16s(a_y + so, tp + y_off, (info & y_bit) != 0);
        }
        cp_async_commit();
    };

    issue(0, prepare());
    issue(1, prepare());
    issue(2, prepare());
    Next nx = prepare();
    for (long long q = 0; q < total; ++q) {
        // tiles q and q + 1 have landed; q - 2's slot is free for q + 3
        cp_async_wait<1>();
        __syncthreads();
        issue(q + 3, nx);
        nx = prepare();
        const Stage& S = st[q % DS];
        const int t = S.meta.x;
        const unsigned info = (unsigned)S.meta.y;
        const float4 c = S.v[tid];
        const float4 f = FIELD ? S.f[tid] : make_float4(Fc, Fc, Fc, Fc);
        const float4 ym = S.v[i_ym];
        const float4 yp = S.v[i_yp];
        // z halos: the previous / next tile of the column (domain faces have none)
        const float4 zm = lz > 0 ? S.v[tid - 16]
                                 : ((info & NB_ZM) ? st[(q + DS - 1) % DS].v[112 + 2 * ly + xh] : c);
        const float4 zp = lz < 7 ? S.v[tid + 16]
                                 : ((info & NB_ZP) ? st[(q + 1) % DS].v[2 * ly + xh] : c);
        const float pcv = reinterpret_cast<const float*>(S.v)[i_pc];
        const float xo = S.xo[tid];
        const float xm0 = xh ? pcv : xo;
        const float xp3 = xh ? xo : pcv;
        float4 o;
        if (info == (NB_ALL | SG_POS)) {
            o = upd4<1, false>(c, f, xm0, xp3, ym, yp, zm, zp, coef, extrap, false, false, false,
                               false, false, false);
        } else if (info == (NB_ALL | SG_NEG)) {
            o = upd4<-1, false>(c, f, xm0, xp3, ym, yp, zm, zp, coef, extrap, false, false, false,
                                false, false, false);
        } else {
            const bool xlo = (xh == 0) && !(info & NB_XM);
            const bool xhi = (xh == 1) && !(info & NB_XP);
            const bool ylo = (ly == 0) && !(info & NB_YM);
            const bool yhi = (ly == 7) && !(info & NB_YP);
            const bool zlo = (lz == 0) && !(info & NB_ZM);
            const bool zhi = (lz == 7) && !(info & NB_ZP);
            o = upd4<0, true>(c, f, xm0, xp3, ym, yp, zm, zp, coef, extrap, xlo, xhi, ylo, yhi,
                              zlo, zhi);
        }
        *reinterpret_cast<float4*>(dst + (size_t)t * TILE_PTS + 4 * tid) = o;
    }
    cp_async_wait<0>();
}

// 8 points per thread: 64-thread CTAs, thread (xh, ly, lzp) owns the quads
// of planes 2 lzp and 2 lzp + 1 (the z neighbour on the other plane is in
// registers), as the list kernel's 8-point variant
template <bool FIELD>
__global__ void __launch_bounds__(64, 16) k_dense2_f32(StepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Stage = DStage<FIELD>;
    Stage* st = reinterpret_cast<Stage*>(smem_raw);
    const int tid = threadIdx.x;
    const int xh = tid & 1, ly = (tid >> 1) & 7, lzp = tid >> 4;
    const int q0 = tid + 16 * lzp, q1 = q0 + 16;
    const int lz0 = 2 * lzp;
    pdl_launch_dependents();
    pdl_wait();
    const Inst in = a.in;
    const int tnx = in.tnx, tny = in.tny, tnz = in.tnz;
    const int ncol = tnx * tny;
    const int G = gridDim.x;
    const int mycols = (int)blockIdx.x < ncol ? (ncol - (int)blockIdx.x + G - 1) / G : 0;
    const long long total = (long long)mycols * tnz;
    if (blockIdx.x == 0 && tid == 0) {
        if (a.updates) atomicAdd(a.updates, (unsigned long long)ncol * tnz * TILE_PTS);
        if (a.updates_timed) atomicAdd(a.updates_timed, (unsigned long long)ncol * tnz * TILE_PTS);
    }
    const float* __restrict__ src = (const float*)a.src;
    float* __restrict__ dst = (float*)a.dst;
    const float* __restrict__ Fp = (const float*)a.F;
    const bool extrap = in.bc == 0;
    const float coef = a.sc->coef;
    const float Fc = (float)in.Fc;
    const unsigned const_sgn = in.Fc >= 0.0 ? SG_POS : SG_NEG;
    const int sy = tnx * TILE_PTS;
    const int x_off0 = xh ? (TILE_PTS + lz0 * 64 + ly * 8) : (-TILE_PTS + lz0 * 64 + ly * 8 + 7);
    const unsigned x_bit = xh ? NB_XP : NB_XM;
    const int y_in = (ly == 0) ? (lz0 * 64 + 56 + 4 * xh) : (lz0 * 64 + 4 * xh);
    const int y_off = ((ly == 0) ? -sy : sy) + y_in;
    const unsigned y_bit = (ly == 0) ? NB_YM : ((ly == 7) ? NB_YP : 0u);
    const int y_slot0 = 128 + ((ly == 7) ? 16 : 0) + 2 * lz0 + xh;
    const int y_slot1 = y_slot0 + 2;
    const int i_ym0 = (ly > 0) ? q0 - 2 : y_slot0;
    const int i_yp0 = (ly < 7) ? q0 + 2 : y_slot0;
    const int i_ym1 = (ly > 0) ? q1 - 2 : y_slot1;
    const int i_yp1 = (ly < 7) ? q1 + 2 : y_slot1;
    const int i_pc0 = 4 * (q0 ^ 1) + (xh ? 3 : 0);
    const int i_pc1 = 4 * (q1 ^ 1) + (xh ? 3 : 0);
    const unsigned sm0 = (unsigned)__cvta_generic_to_shared(st);
    constexpr unsigned SB = (unsigned)sizeof(Stage);
    const unsigned a_c0 = sm0 + (unsigned)offsetof(Stage, v) + 16u * q0;
    const unsigned a_f0 = sm0 + (unsigned)offsetof(Stage, f) + 16u * q0;
    const unsigned a_x0 = sm0 + (unsigned)offsetof(Stage, xo) + 4u * q0;
    const unsigned a_y0 = sm0 + (unsigned)offsetof(Stage, v) + 16u * y_slot0;

    struct Next {
        long long t;
        unsigned info;
    };
    int pci = 0, ptz = 0, pcol = (int)blockIdx.x;
    int pty = pcol / tnx, ptx = pcol - pty * tnx;
    auto prepare = [&]() {
        Next nx{0, 0u};
        if (pci < mycols) {
            nx.t = (long long)ptz * ncol + pcol;
            unsigned nb = 0;
            if (ptx > 0) nb |= NB_XM;
            if (ptx < tnx - 1) nb |= NB_XP;
            if (pty > 0) nb |= NB_YM;
            if (pty < tny - 1) nb |= NB_YP;
            if (ptz > 0) nb |= NB_ZM;
            if (ptz < tnz - 1) nb |= NB_ZP;
            nx.info = nb | (a.tile_sgn ? (unsigned)__ldg(a.tile_sgn + nx.t) : const_sgn);
            if (++ptz == tnz) {
                ptz = 0;
                ++pci;
                pcol += G;
                pty = pcol / tnx;
                ptx = pcol - pty * tnx;
            }
        }
        return nx;
    };
    auto issue = [&](long long q, const Next& nx) {
        if (q < total) {
            const int s = (int)(q % DS);
            const unsigned so = (unsigned)s * SB;
            const float* tp = src + nx.t * TILE_PTS;
            if (tid == 0) st[s].meta = make_int4((int)nx.t, (int)nx.info, 0, 0);
            cp_async16s(a_c0 + so, tp + 4 * q0);
            cp_async16s(a_c0 + so + 256u, tp + 4 * q1);
            if (FIELD) {
                cp_async16s(a_f0 + so, Fp + nx.t * TILE_PTS + 4 * q0);
                cp_async16s(a_f0 + so + 256u, Fp + nx.t * TILE_PTS + 4 * q1);
            }
            const bool px = (nx.info & x_bit) != 0, py = (nx.info & y_bit) != 0;
            cp_async4s(a_x0 + so, tp + x_off0, px);
            cp_async4s(a_x0 + so + 64u, tp + x_off0 + 64, px);
            cp_async16s(a_y0 + so, tp + y_off, py);
            cp_async16s(a_y0 + so + 32u, tp + y_off + 64, py);
        }
        cp_async_commit();
    };

    issue(0, prepare());
    issue(1, prepare());
    issue(2, prepare());
    Next nx = prepare();
    for (long long q = 0; q < total; ++q) {
        cp_async_wait<1>();
        __syncthreads();
        issue(q + 3, nx);
        nx = prepare();
        const Stage& S = st[q % DS];
        const int t = S.meta.x;
        const unsigned info = (unsigned)S.meta.y;
        const float4 c0 = S.v[q0], c1 = S.v[q1];
        const float4 f0 = FIELD ? S.f[q0] : make_float4(Fc, Fc, Fc, Fc);
        const float4 f1 = FIELD ? S.f[q1] : make_float4(Fc, Fc, Fc, Fc);
        const float4 ym0 = S.v[i_ym0], yp0 = S.v[i_yp0];
        const float4 ym1 = S.v[i_ym1], yp1 = S.v[i_yp1];
        const float4 zm0 = lzp > 0 ? S.v[q0 - 16]
                                   : ((info & NB_ZM) ? st[(q + DS - 1) % DS].v[112 + 2 * ly + xh] : c0);
        const float4 zp1 = lzp < 3 ? S.v[q1 + 16]
                                   : ((info & NB_ZP) ? st[(q + 1) % DS].v[2 * ly + xh] : c1);
        const float pc0 = reinterpret_cast<const float*>(S.v)[i_pc0];
        const float pc1 = reinterpret_cast<const float*>(S.v)[i_pc1];
        const float xo0 = S.xo[q0], xo1 = S.xo[q1];
        const float xm0a = xh ? pc0 : xo0, xp3a = xh ? xo0 : pc0;
        const float xm0b = xh ? pc1 : xo1, xp3b = xh ? xo1 : pc1;
        float4 o0, o1;
        if (info == (NB_ALL | SG_POS)) {
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
        float* dp = dst + (size_t)t * TILE_PTS;
        *reinterpret_cast<float4*>(dp + 4 * q0) = o0;
        *reinterpret_cast<float4*>(dp + 4 * q1) = o1;
    }
    cp_async_wait<0>();
}

template <typename K>
int dense_grid(K kernel, size_t smem, int ncol, int threads)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
    if (per < 1) per = 1;
    const int g = sms * per;
    return g < ncol ? g : ncol;
}

template <bool FIELD, int PPT>
cudaError_t launch_dense(const StepArgs& a, int grid_pct, cudaStream_t s)
{
    constexpr size_t smem = sizeof(DStage<FIELD>) * DS;
    constexpr int threads = PPT == 8 ? 64 : 128;
    auto kernel = PPT == 8 ? k_dense2_f32<FIELD> : k_dense_f32<FIELD>;
    static int full = 0;
    if (!full) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        full = dense_grid(kernel, smem, 1 << 30, threads);
    }
    const int ncol = a.in.tnx * a.in.tny;
    int grid = (int)((long long)full * grid_pct / 100);
    if (grid < 1) grid = 1;
    if (grid > ncol) grid = ncol;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

}  // namespace

cudaError_t launch_dense_step(const StepArgs& a, const StepConfig& cfg, cudaStream_t s)
{
    if (a.list_inst || a.op != OP_PLAIN || a.core) return cudaErrorInvalidValue;
    if (cfg.ppt == 8)
        return a.F ? launch_dense<true, 8>(a, cfg.grid_pct, s) : launch_dense<false, 8>(a, cfg.grid_pct, s);
    return a.F ? launch_dense<true, 4>(a, cfg.grid_pct, s) : launch_dense<false, 4>(a, cfg.grid_pct, s);
}

}  // namespace lsk
