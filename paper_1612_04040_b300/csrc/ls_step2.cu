// ls_step2.cu -- two upwind steps (Eq. 3-5 of section 1) per pass over the
// active tiles (temporal blocking; FP32, single grid, plain scheme).
//
// One persistent CTA of 128 threads takes one active 8^3 tile at a time.  It
// stages phi^n of the tile, of depth-2 slabs of its six face neighbours and
// of the twelve 1-deep edge lines next to them, computes the intermediate
// phi' (one step) on the tile and on the one-cell face layers around it --
// the face layer of an inactive neighbour keeps phi^n (frozen), as in the
// one-step kernel -- and then phi^{n+2} on the tile from phi'.  Every point
// goes through the same per-point arithmetic as the one-step kernel, so two
// steps here give the bits of two one-step launches; a pass moves 12 bytes
// per tile point (F field) for two updates instead of 24, at the price of
// the face-layer points computed twice (896 intermediate updates for 512).
// The list entry's face-neighbour bits (which neighbours are active) come
// from the rebuild.  Two-stage cp.async ring (the next tile's loads overlap
// this tile's arithmetic).
#include <cstddef>

#include "ls_internal.cuh"
#include "ls_stencil.cuh"

namespace lsk {

namespace {

// phi^n staged: z, y in [-2, 10), x in [-4, 12) (x padded so that tile rows
// start on 16 bytes); phi': z, y in [-1, 9), x in [-4, 12)
constexpr int PX = 16, PY = 12, PZ = 12;
constexpr int QY = 10, QZ = 10;
__device__ __forceinline__ int pidx(int z, int y, int x) { return ((z + 2) * PY + (y + 2)) * PX + (x + 4); }
__device__ __forceinline__ int qidx(int z, int y, int x) { return ((z + 1) * QY + (y + 1)) * PX + (x + 4); }

template <bool FIELD>
struct Stage2 {
    float P[PZ * PY * PX];       // phi^n, tile + depth-2 face slabs + edge lines
    float4 Ft[FIELD ? 128 : 1];  // F on the tile
    float Ff[FIELD ? 6 * 64 : 1];  // F on the six face layers: x-, x+ [z*8+y];
                                   // y-, y+ [z*8+x]; z-, z+ [y*8+x]
    int4 meta;                   // tile id, info byte, active face neighbours
};

// one face-layer point of the intermediate step: c and its six neighbours,
// the missing ones (domain faces) replaced by the face rule
__device__ __forceinline__ float layer_point(float c, float f, float xm, float xp, float ym, float yp,
                                             float zm, float zp, bool xlo, bool xhi, bool ylo,
                                             bool yhi, bool zlo, bool zhi, bool extrap, float coef)
{
    float dmx = c - xm, dpx = xp - c;
    float dmy = c - ym, dpy = yp - c;
    float dmz = c - zm, dpz = zp - c;
    if (xlo) dmx = extrap ? dpx : 0.f;
    if (xhi) dpx = extrap ? dmx : 0.f;
    if (ylo) dmy = extrap ? dpy : 0.f;
    if (yhi) dpy = extrap ? dmy : 0.f;
    if (zlo) dmz = extrap ? dpz : 0.f;
    if (zhi) dpz = extrap ? dmz : 0.f;
    return upd32<0>(c, f, dmx, dpx, dmy, dpy, dmz, dpz, coef);
}

template <bool FIELD, bool CLASSIFY>
__global__ void __launch_bounds__(128, 6) k_step2_f32(StepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Stage = Stage2<FIELD>;
    Stage* st = reinterpret_cast<Stage*>(smem_raw);
    float* Q = reinterpret_cast<float*>(st + 2);   // phi', QZ * QY * PX floats
    __shared__ unsigned smin[2];
    const int tid = threadIdx.x;
    const int xh = tid & 1, ly = (tid >> 1) & 7, lz = tid >> 4;
    pdl_launch_dependents();
    pdl_wait();
    const int n = *a.count;
    if (blockIdx.x == 0 && tid == 0) {
        if (a.updates) atomicAdd(a.updates, 2ull * (unsigned long long)n * TILE_PTS);
        if (a.updates_timed) atomicAdd(a.updates_timed, 2ull * (unsigned long long)n * TILE_PTS);
        if (a.updates2) atomicAdd(a.updates2, (unsigned long long)n * TILE_PTS);
    }
    const bool rev = a.reverse != 0;
    auto ent = [&](int k) { return rev ? n - 1 - k : k; };
    const float* __restrict__ src = (const float*)a.src;
    float* __restrict__ dst = (float*)a.dst;
    const float* __restrict__ Fp = (const float*)a.F;
    const bool extrap = a.in.bc == 0;
    const float coef = a.sc->coef;
    const float Fc = (float)a.in.Fc;
    const double gamma = a.in.gamma;
    const long long sy = (long long)a.in.tnx * TILE_PTS;
    const long long sz = (long long)a.in.tnx * a.in.tny * TILE_PTS;
    const int stride = gridDim.x;

    // stage list entry kk (tile t, info, active neighbours) into slot s
    auto issue = [&](unsigned t, unsigned info, unsigned nact, int s) {
        Stage& S = st[s];
        const float* tp = src + (size_t)t * TILE_PTS;
        const unsigned sP = (unsigned)__cvta_generic_to_shared(S.P);
        if (tid == 0) {
            S.meta = make_int4((int)t, (int)info, (int)nact, 0);
            if (CLASSIFY) smin[s] = 0x7f800000u;
        }
        const bool XM = info & NB_XM, XP = info & NB_XP, YM = info & NB_YM, YP = info & NB_YP;
        const bool ZM = info & NB_ZM, ZP = info & NB_ZP;
        // (1) the tile
        cp_async16s(sP + 4u * pidx(lz, ly, 4 * xh), tp + 4 * tid);
        // (2) F on the tile
        if (FIELD) {
            cp_async16s((unsigned)__cvta_generic_to_shared(&S.Ft[tid]), Fp + (size_t)t * TILE_PTS + 4 * tid);
        }
        // (3) x slabs, depth 2 (8 bytes per row)
        {
            const int r = tid & 63, z = r >> 3, y = r & 7;
            if (tid < 64)
                cp_async8s(sP + 4u * pidx(z, y, -2), tp - TILE_PTS + z * 64 + y * 8 + 6, XM);
            else
                cp_async8s(sP + 4u * pidx(z, y, 8), tp + TILE_PTS + z * 64 + y * 8, XP);
        }
        // (4) y slabs (tid < 64) and z slabs, depth 2 (16 bytes per half row)
        if (tid < 64) {
            const int j = tid, side = j >> 5, z = (j >> 2) & 7, row = (j >> 1) & 1, half = j & 1;
            if (side == 0)
                cp_async16s(sP + 4u * pidx(z, -2 + row, 4 * half), tp - sy + z * 64 + (6 + row) * 8 + 4 * half, YM);
            else
                cp_async16s(sP + 4u * pidx(z, 8 + row, 4 * half), tp + sy + z * 64 + row * 8 + 4 * half, YP);
        } else {
            const int j = tid - 64, side = j >> 5, p = (j >> 4) & 1, y = (j >> 1) & 7, half = j & 1;
            if (side == 0)
                cp_async16s(sP + 4u * pidx(-2 + p, y, 4 * half), tp - sz + (6 + p) * 64 + y * 8 + 4 * half, ZM);
            else
                cp_async16s(sP + 4u * pidx(8 + p, y, 4 * half), tp + sz + p * 64 + y * 8 + 4 * half, ZP);
        }
        // (5) the twelve edge lines next to the face layers
        if (tid < 32) {  // x-y edges, along z
            const int e = tid >> 3, z = tid & 7, sx = e & 1, sgy = e >> 1;
            const long long off = (sx ? TILE_PTS : -TILE_PTS) + (sgy ? sy : -sy) + z * 64 + (sgy ? 0 : 56) + (sx ? 0 : 7);
            cp_async4s(sP + 4u * pidx(z, sgy ? 8 : -1, sx ? 8 : -1), tp + off, (sx ? XP : XM) && (sgy ? YP : YM));
        } else if (tid < 64) {  // x-z edges, along y
            const int j = tid - 32, e = j >> 3, y = j & 7, sx = e & 1, sgz = e >> 1;
            const long long off = (sx ? TILE_PTS : -TILE_PTS) + (sgz ? sz : -sz) + (sgz ? 0 : 448) + y * 8 + (sx ? 0 : 7);
            cp_async4s(sP + 4u * pidx(sgz ? 8 : -1, y, sx ? 8 : -1), tp + off, (sx ? XP : XM) && (sgz ? ZP : ZM));
        } else if (tid < 72) {  // y-z edges, along x (16 bytes per half)
            const int j = tid - 64, e = j >> 1, half = j & 1, sgy = e & 1, sgz = e >> 1;
            const long long off = (sgy ? sy : -sy) + (sgz ? sz : -sz) + (sgz ? 0 : 448) + (sgy ? 0 : 56) + 4 * half;
            cp_async16s(sP + 4u * pidx(sgz ? 8 : -1, sgy ? 8 : -1, 4 * half), tp + off,
                        (sgy ? YP : YM) && (sgz ? ZP : ZM));
        }
        // (6) F on the face layers
        if (FIELD) {
            const unsigned sF = (unsigned)__cvta_generic_to_shared(S.Ff);
            const float* fp = Fp + (size_t)t * TILE_PTS;
            {
                const int face = tid >> 6, i = tid & 63, z = i >> 3, y = i & 7;
                const long long off = face ? (TILE_PTS + z * 64 + y * 8) : (-TILE_PTS + z * 64 + y * 8 + 7);
                cp_async4s(sF + 4u * (face * 64 + i), fp + off, face ? XP : XM);
            }
            if (tid < 64) {
                const int face = 2 + (tid >> 4), q = tid & 15, u = q >> 1, half = q & 1;
                long long off;
                bool ok;
                if (face == 2) { off = -sy + u * 64 + 56 + 4 * half; ok = YM; }
                else if (face == 3) { off = sy + u * 64 + 4 * half; ok = YP; }
                else if (face == 4) { off = -sz + 448 + u * 8 + 4 * half; ok = ZM; }
                else { off = sz + u * 8 + 4 * half; ok = ZP; }
                cp_async16s(sF + 4u * (face * 64 + u * 8 + 4 * half), fp + off, ok);
            }
        }
    };
    auto fetch = [&](int k, unsigned& t, unsigned& info, unsigned& nact) {
        k = ent(k);
        t = (unsigned)__ldg(a.list + k);
        info = __ldg(a.info + k);
        nact = __ldg(a.nact + k);
    };

    int kn = blockIdx.x;
    if (kn < n) {
        unsigned t, info, nact;
        fetch(kn, t, info, nact);
        issue(t, info, nact, 0);
    }
    cp_async_commit();
    kn += stride;
    unsigned t1 = 0, i1 = 0, a1 = 0;
    if (kn < n) fetch(kn, t1, i1, a1);
    int cur = 0, prev = -1, prev_t = -1;
    for (int k = blockIdx.x; k < n; k += stride) {
        // this entry's stage has landed; every thread is done with the other
        // slot (the previous entry), which now receives the next entry
        cp_async_wait<0>();
        __syncthreads();
        if (CLASSIFY && tid == 0 && prev >= 0)
            a.core[prev_t] = ((double)__uint_as_float(smin[prev]) < gamma) ? 1 : 0;
        if (kn < n) issue(t1, i1, a1, cur ^ 1);
        cp_async_commit();
        kn += stride;
        if (kn < n) fetch(kn, t1, i1, a1);

        const Stage& S = st[cur];
        const float* P = S.P;
        const int t = S.meta.x;
        const unsigned info = (unsigned)S.meta.y;
        const unsigned nact = (unsigned)S.meta.z;
        const bool XM = info & NB_XM, XP = info & NB_XP, YM = info & NB_YM, YP = info & NB_YP;
        const bool ZM = info & NB_ZM, ZP = info & NB_ZP;
        const int x0 = 4 * xh;
        const bool xlo = xh == 0 && !XM, xhi = xh == 1 && !XP;
        const bool ylo = ly == 0 && !YM, yhi = ly == 7 && !YP;
        const bool zlo = lz == 0 && !ZM, zhi = lz == 7 && !ZP;

        // ---- intermediate step: the tile's own points
        {
            const float4 c = *reinterpret_cast<const float4*>(P + pidx(lz, ly, x0));
            const float4 f = FIELD ? S.Ft[tid] : make_float4(Fc, Fc, Fc, Fc);
            const float xm = P[pidx(lz, ly, x0 - 1)], xp = P[pidx(lz, ly, x0 + 4)];
            const float4 ym = *reinterpret_cast<const float4*>(P + pidx(lz, ly - 1, x0));
            const float4 yp = *reinterpret_cast<const float4*>(P + pidx(lz, ly + 1, x0));
            const float4 zm = *reinterpret_cast<const float4*>(P + pidx(lz - 1, ly, x0));
            const float4 zp = *reinterpret_cast<const float4*>(P + pidx(lz + 1, ly, x0));
            float4 o;
            if (info == (NB_ALL | SG_POS))
                o = upd4<1, false>(c, f, xm, xp, ym, yp, zm, zp, coef, extrap, false, false, false, false, false, false);
            else if (info == (NB_ALL | SG_NEG))
                o = upd4<-1, false>(c, f, xm, xp, ym, yp, zm, zp, coef, extrap, false, false, false, false, false, false);
            else
                o = upd4<0, true>(c, f, xm, xp, ym, yp, zm, zp, coef, extrap, xlo, xhi, ylo, yhi, zlo, zhi);
            *reinterpret_cast<float4*>(Q + qidx(lz, ly, x0)) = o;
        }
        // ---- intermediate step: one point of each pair of face layers.
        // A face layer of an active neighbour advances, of an inactive one
        // keeps phi^n (frozen), of a missing one (domain face) is not needed.
        {
            const int side = tid >> 6, i = tid & 63, u = i >> 3, v = i & 7;
            // x layer at x = -1 / 8, point (z, y) = (u, v)
            {
                const bool has = side ? XP : XM;
                const unsigned bit = side ? NB_XP : NB_XM;
                const int x = side ? 8 : -1, z = u, y = v;
                if (has) {
                    const float c = P[pidx(z, y, x)];
                    float r = c;
                    if (nact & bit) {
                        const float f = FIELD ? S.Ff[side * 64 + i] : Fc;
                        const bool fylo = y == 0 && !YM, fyhi = y == 7 && !YP;
                        const bool fzlo = z == 0 && !ZM, fzhi = z == 7 && !ZP;
                        r = layer_point(c, f, P[pidx(z, y, x - 1)], P[pidx(z, y, x + 1)],
                                        fylo ? c : P[pidx(z, y - 1, x)], fyhi ? c : P[pidx(z, y + 1, x)],
                                        fzlo ? c : P[pidx(z - 1, y, x)], fzhi ? c : P[pidx(z + 1, y, x)],
                                        false, false, fylo, fyhi, fzlo, fzhi, extrap, coef);
                    }
                    Q[qidx(z, y, x)] = r;
                }
            }
            // y layer at y = -1 / 8, point (z, x) = (u, v)
            {
                const bool has = side ? YP : YM;
                const unsigned bit = side ? NB_YP : NB_YM;
                const int y = side ? 8 : -1, z = u, x = v;
                if (has) {
                    const float c = P[pidx(z, y, x)];
                    float r = c;
                    if (nact & bit) {
                        const float f = FIELD ? S.Ff[(2 + side) * 64 + i] : Fc;
                        const bool fxlo = x == 0 && !XM, fxhi = x == 7 && !XP;
                        const bool fzlo = z == 0 && !ZM, fzhi = z == 7 && !ZP;
                        r = layer_point(c, f, fxlo ? c : P[pidx(z, y, x - 1)], fxhi ? c : P[pidx(z, y, x + 1)],
                                        P[pidx(z, y - 1, x)], P[pidx(z, y + 1, x)],
                                        fzlo ? c : P[pidx(z - 1, y, x)], fzhi ? c : P[pidx(z + 1, y, x)],
                                        fxlo, fxhi, false, false, fzlo, fzhi, extrap, coef);
                    }
                    Q[qidx(z, y, x)] = r;
                }
            }
            // z layer at z = -1 / 8, point (y, x) = (u, v)
            {
                const bool has = side ? ZP : ZM;
                const unsigned bit = side ? NB_ZP : NB_ZM;
                const int z = side ? 8 : -1, y = u, x = v;
                if (has) {
                    const float c = P[pidx(z, y, x)];
                    float r = c;
                    if (nact & bit) {
                        const float f = FIELD ? S.Ff[(4 + side) * 64 + i] : Fc;
                        const bool fxlo = x == 0 && !XM, fxhi = x == 7 && !XP;
                        const bool fylo = y == 0 && !YM, fyhi = y == 7 && !YP;
                        r = layer_point(c, f, fxlo ? c : P[pidx(z, y, x - 1)], fxhi ? c : P[pidx(z, y, x + 1)],
                                        fylo ? c : P[pidx(z, y - 1, x)], fyhi ? c : P[pidx(z, y + 1, x)],
                                        P[pidx(z - 1, y, x)], P[pidx(z + 1, y, x)],
                                        fxlo, fxhi, fylo, fyhi, false, false, extrap, coef);
                    }
                    Q[qidx(z, y, x)] = r;
                }
            }
        }
        __syncthreads();
        // ---- second step on the tile, from phi'
        {
            const float4 c = *reinterpret_cast<const float4*>(Q + qidx(lz, ly, x0));
            const float4 f = FIELD ? S.Ft[tid] : make_float4(Fc, Fc, Fc, Fc);
            const float xm = Q[qidx(lz, ly, x0 - 1)], xp = Q[qidx(lz, ly, x0 + 4)];
            const float4 ym = *reinterpret_cast<const float4*>(Q + qidx(lz, ly - 1, x0));
            const float4 yp = *reinterpret_cast<const float4*>(Q + qidx(lz, ly + 1, x0));
            const float4 zm = *reinterpret_cast<const float4*>(Q + qidx(lz - 1, ly, x0));
            const float4 zp = *reinterpret_cast<const float4*>(Q + qidx(lz + 1, ly, x0));
            float4 o;
            if (info == (NB_ALL | SG_POS))
                o = upd4<1, false>(c, f, xm, xp, ym, yp, zm, zp, coef, extrap, false, false, false, false, false, false);
            else if (info == (NB_ALL | SG_NEG))
                o = upd4<-1, false>(c, f, xm, xp, ym, yp, zm, zp, coef, extrap, false, false, false, false, false, false);
            else
                o = upd4<0, true>(c, f, xm, xp, ym, yp, zm, zp, coef, extrap, xlo, xhi, ylo, yhi, zlo, zhi);
            *reinterpret_cast<float4*>(dst + (size_t)t * TILE_PTS + 4 * tid) = o;
            if (CLASSIFY) {
                const float mn = fminf(fminf(fabsf(o.x), fabsf(o.y)), fminf(fabsf(o.z), fabsf(o.w)));
                const unsigned wm = __reduce_min_sync(0xffffffffu, __float_as_uint(mn));
                if ((tid & 31) == 0) atomicMin(&smin[cur], wm);
            }
        }
        prev = cur;
        prev_t = t;
        cur ^= 1;
    }
    if (CLASSIFY) {
        __syncthreads();
        if (tid == 0 && prev >= 0)
            a.core[prev_t] = ((double)__uint_as_float(smin[prev]) < gamma) ? 1 : 0;
    }
    cp_async_wait<0>();
}

template <typename K>
int occupancy_grid2(K kernel, size_t smem)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 128, smem);
    if (per < 1) per = 1;
    return sms * per;
}

template <bool FIELD, bool CLS>
cudaError_t launch2(const StepArgs& a, int grid_pct, cudaStream_t s)
{
    constexpr size_t smem = 2 * sizeof(Stage2<FIELD>) + sizeof(float) * QZ * QY * PX;
    static int full = 0;
    if (!full) {
        cudaError_t e = cudaFuncSetAttribute(k_step2_f32<FIELD, CLS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        full = occupancy_grid2(k_step2_f32<FIELD, CLS>, smem);
    }
    int grid = (int)((long long)full * grid_pct / 100);
    if (grid < 1) grid = 1;
    if (a.max_grid > 0 && grid > a.max_grid) grid = a.max_grid;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_step2_f32<FIELD, CLS>, a);
}

}  // namespace

cudaError_t launch_step2(const StepArgs& a, const StepConfig& cfg, cudaStream_t s)
{
    if (a.list_inst || !a.nact || a.op != OP_PLAIN) return cudaErrorInvalidValue;
    const bool field = a.F != nullptr, cls = a.core != nullptr;
    const int pct = cfg.grid_pct2;
    if (field) return cls ? launch2<true, true>(a, pct, s) : launch2<true, false>(a, pct, s);
    return cls ? launch2<false, true>(a, pct, s) : launch2<false, false>(a, pct, s);
}

}  // namespace lsk
