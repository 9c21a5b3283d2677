// ls_band.cu -- band rebuild kernels (section 1.1, Step 1 and Eq. 6 / 11),
// the active-tile compaction (the "active points array" of section 2, here
// at tile granularity), the max|F| reduction behind the CFL time step, and
// the row-major <-> bricked layout conversion.
//
// All band decisions are exact: min |phi| over a tile is exact in any
// precision, and the tube test min|phi| < gamma is done in FP64 against
// gamma = halfwidth * h computed in FP64 on the host.
#include <cuda/atomic>
#include <utility>

#include "ls_internal.cuh"
#include "ls_stencil.cuh"

namespace lsk {

namespace {

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// The rebuild kernels that follow a stencil launch (dilate) or another
// rebuild kernel (scatter) are launched with programmatic stream
// serialisation: their CTAs are scheduled as the previous grid drains and
// wait (pdl_wait, their first statement) for its completion and memory.
template <typename... KArgs, typename... Args>
cudaError_t launch_after(void (*kernel)(KArgs...), int grid, int block, cudaStream_t s,
                         Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename T>
__device__ __forceinline__ bool finite_val(T v) { return isfinite(v); }

// ---------------------------------------------------------------------------
// layout conversion: one 128-thread block per tile; thread -> 4 x-consecutive
// points (lz, ly, 4*xh .. 4*xh+3), i.e. element offset 4*threadIdx.x
// ---------------------------------------------------------------------------
template <typename T, bool PACK>
__global__ void __launch_bounds__(128) k_convert(const T* __restrict__ src, T* __restrict__ dst,
                                                 Inst in, unsigned* nonfinite)
{
    const int tid = threadIdx.x;
    const int xh = tid & 1, ly = (tid >> 1) & 7, lz = tid >> 4;
    const long long tpl = (long long)in.tnx * in.tny;
    for (long long t = blockIdx.x; t < in.ntiles; t += gridDim.x) {
        const int tz = (int)(t / tpl);
        const int rem = (int)(t - (long long)tz * tpl);
        const int ty = rem / in.tnx, tx = rem - ty * in.tnx;
        const size_t rm = ((size_t)(tz * TILE + lz) * in.ny + (size_t)(ty * TILE + ly)) * in.nx
                          + (size_t)(tx * TILE + 4 * xh);
        const size_t bk = (size_t)t * TILE_PTS + 4 * tid;
        const size_t from = PACK ? rm : bk;
        const size_t to = PACK ? bk : rm;
        T v0, v1, v2, v3;
        if constexpr (sizeof(T) == 4) {
            const float4 v = *reinterpret_cast<const float4*>(src + from);
            v0 = v.x; v1 = v.y; v2 = v.z; v3 = v.w;
            *reinterpret_cast<float4*>(dst + to) = v;
        } else {
            const double2 a = *reinterpret_cast<const double2*>(src + from);
            const double2 b = *reinterpret_cast<const double2*>(src + from + 2);
            v0 = a.x; v1 = a.y; v2 = b.x; v3 = b.y;
            *reinterpret_cast<double2*>(dst + to) = a;
            *reinterpret_cast<double2*>(dst + to + 2) = b;
        }
        if (PACK && nonfinite) {
            const bool bad = !(finite_val(v0) && finite_val(v1) && finite_val(v2) && finite_val(v3));
            if (bad) *nonfinite = 1u;  // a flag (host-mapped memory): any writer sets it
        }
    }
}

// ---------------------------------------------------------------------------
// per-tile reductions: one warp per tile
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_min(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ const Inst& inst_of(long long t, const Inst* d_inst,
                                               const uint16_t* tile_inst, const Inst& single)
{
    return tile_inst ? d_inst[tile_inst[t]] : single;
}

// max |v| over the 512 values of a tile, by one warp
template <typename T>
__device__ __forceinline__ T tile_absmax(const T* __restrict__ p)
{
    T m = T(0);
    if constexpr (sizeof(T) == 4) {
        const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 v = __ldg(q + lane_id() + 32 * k);
            m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
    } else {
        const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const double2 v = __ldg(q + lane_id() + 32 * k);
            m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
        }
    }
    return warp_max(m);
}

// min |v| over the 512 values of a tile, by one warp
template <typename T>
__device__ __forceinline__ T tile_absmin(const T* __restrict__ p)
{
    T m;
    if constexpr (sizeof(T) == 4) {
        m = __int_as_float(0x7f800000);
        const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 v = __ldg(q + lane_id() + 32 * k);
            m = fminf(m, fminf(fminf(fabsf(v.x), fabsf(v.y)), fminf(fabsf(v.z), fabsf(v.w))));
        }
    } else {
        m = __longlong_as_double(0x7ff0000000000000ll);
        const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const double2 v = __ldg(q + lane_id() + 32 * k);
            m = fmin(m, fmin(fabs(v.x), fabs(v.y)));
        }
    }
    return warp_min(m);
}

// per tile: max |F| (for the CFL bound) and the sign code of its speeds
template <typename T>
__global__ void __launch_bounds__(256) k_tile_speed(const T* __restrict__ F, T* __restrict__ out,
                                                    uint8_t* sgn, long long ntiles)
{
    const long long warps = (long long)gridDim.x * 8;
    for (long long t = (long long)blockIdx.x * 8 + (threadIdx.x >> 5); t < ntiles; t += warps) {
        const T* p = F + (size_t)t * TILE_PTS;
        const T m = tile_absmax(p);
        bool pos = true, neg = true;
        for (int k = lane_id(); k < TILE_PTS; k += 32) {
            const T v = __ldg(p + k);
            pos = pos && (v >= T(0));
            neg = neg && (v < T(0));
        }
        pos = __all_sync(0xffffffffu, pos);
        neg = __all_sync(0xffffffffu, neg);
        if (lane_id() == 0) {
            out[t] = m;
            sgn[t] = (uint8_t)(pos ? SG_POS : (neg ? SG_NEG : 0u));
        }
    }
}

// neighbour-existence bits of tile t (single instance or batched table)
__device__ __forceinline__ unsigned nb_bits(long long t, const Inst& in)
{
    const int loc = (int)(t - in.tile_base);  // < 2^31 tiles per instance
    const int tpl = in.tnx * in.tny;
    const int tz = loc / tpl;
    const int rem = loc - tz * tpl;
    const int ty = rem / in.tnx, tx = rem - ty * in.tnx;
    unsigned b = 0;
    if (tx > 0) b |= NB_XM;
    if (tx < in.tnx - 1) b |= NB_XP;
    if (ty > 0) b |= NB_YM;
    if (ty < in.tny - 1) b |= NB_YP;
    if (tz > 0) b |= NB_ZM;
    if (tz < in.tnz - 1) b |= NB_ZP;
    return b;
}

// Eq. 6 per tile: core = (min |phi| over the tile) < gamma, compared in FP64
template <typename T>
__global__ void __launch_bounds__(256) k_classify_all(const T* __restrict__ phi, uint8_t* core,
                                                      const Inst* d_inst,
                                                      const uint16_t* tile_inst, Inst single,
                                                      long long ntiles)
{
    const long long warps = (long long)gridDim.x * 8;
    for (long long t = (long long)blockIdx.x * 8 + (threadIdx.x >> 5); t < ntiles; t += warps) {
        const T m = tile_absmin(phi + (size_t)t * TILE_PTS);
        if (lane_id() == 0) {
            const double g = inst_of(t, d_inst, tile_inst, single).gamma;
            core[t] = ((double)m < g) ? 1 : 0;
        }
    }
}

// ---------------------------------------------------------------------------
// dilation by one tile (26 neighbours, inside the instance) and per-block
// active counts.  One thread per tile, 256 per block.  act[t] keeps the new
// flag in bit 0 and the previous one in bit 1 (the scatter pass uses both to
// find the tiles that leave the active set).
// ---------------------------------------------------------------------------
// The block that finishes last (every block's thread 0 releases its writes
// when it counts itself) sees the results of all blocks; true in all its
// threads.
// That block resets the counter for the next launch.  No block waits.
__device__ __forceinline__ bool last_block(unsigned* done)
{
    // what the last block reads of the other blocks (their count, their max
    // |F| bits) is written by each block's thread 0, so only that thread
    // orders its writes before the counter moves (release) and the last one
    // orders its reads after it (acquire); the other threads wait at the
    // barrier instead of at a fence of their own
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> d(*done);
        last = d.fetch_add(1u, cuda::memory_order_acq_rel) == gridDim.x - 1;
        if (last) d.store(0u, cuda::memory_order_relaxed);
    }
    __syncthreads();
    return last;
}

// exclusive scan in place of n block counts by one 256-thread block (the
// counts of other blocks are read from L2); total -> *total
__device__ void block_scan256(int* counts, int n, int* total)
{
    __shared__ int warp_sums[8];
    const int per = (n + 255) / 256;
    const int b0 = threadIdx.x * per;
    int local = 0;
    for (int k = 0; k < per; ++k)
        if (b0 + k < n) local += __ldcg(counts + b0 + k);
    int v = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if ((int)lane_id() >= o) v += u;
    }
    if (lane_id() == 31) warp_sums[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        int w = threadIdx.x < 8 ? warp_sums[threadIdx.x] : 0;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, w, o);
            if ((int)threadIdx.x >= o) w += u;
        }
        if (threadIdx.x < 8) warp_sums[threadIdx.x] = w;
    }
    __syncthreads();
    int run = v - local + ((threadIdx.x >> 5) ? warp_sums[(threadIdx.x >> 5) - 1] : 0);
    for (int k = 0; k < per; ++k) {
        if (b0 + k < n) {
            const int c = __ldcg(counts + b0 + k);
            counts[b0 + k] = run;
            run += c;
        }
    }
    if (threadIdx.x == 255) *total = run;
}

__global__ void __launch_bounds__(256) k_dilate(const uint8_t* __restrict__ core, uint8_t* act,
                                                int* block_counts, const Inst* d_inst,
                                                const uint16_t* tile_inst, Inst single,
                                                long long ntiles, unsigned* done, int* total,
                                                int conn)
{
    pdl_wait();
    const long long t = (long long)blockIdx.x * 256 + threadIdx.x;
    int on = 0;
    if (t < ntiles) {
        const Inst& in = inst_of(t, d_inst, tile_inst, single);
        // tile ids of one instance fit in 32 bits (the active list is int)
        const int loc = (int)(t - in.tile_base);
        const int tpl = in.tnx * in.tny;
        const int tz = loc / tpl;
        const int rem = loc - tz * tpl;
        const int ty = rem / in.tnx, tx = rem - ty * in.tnx;
        const uint8_t* ct = core + t;
        // which neighbours exist, per axis and side; a neighbour is read when
        // its three axis tests hold (and, with 6-connectivity, when it is a
        // face neighbour).  All 27 (or 7) flags are loaded independently,
        // then OR-ed: no chain of dependent loads; the offsets are the row
        // pointers' plus a constant.
        const bool ex[3] = {tx > 0, true, tx < in.tnx - 1};
        const bool ey[3] = {ty > 0, true, ty < in.tny - 1};
        const bool ez[3] = {tz > 0, true, tz < in.tnz - 1};
        const bool all26 = conn != 6;
        unsigned acc = 0;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const uint8_t* row = ct + (long long)dz * tpl + (long long)dy * in.tnx;
                const bool vzy = ez[dz + 1] && ey[dy + 1];
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const bool face = abs(dx) + abs(dy) + abs(dz) <= 1;
                    if (vzy && ex[dx + 1] && (face || all26)) acc |= row[dx];
                }
            }
        }
        on = acc != 0;
        // a ghost row (a neighbour slab's copy) is never active here
        if (((in.ghost & 1) && tz == 0) || ((in.ghost & 2) && tz == in.tnz - 1)) on = 0;
        const int old = act[t] & 1;
        act[t] = (uint8_t)(on | (old << 1));
    }
    const int cnt = __syncthreads_count(on);
    if (threadIdx.x == 0) block_counts[blockIdx.x] = cnt;
    // the last block turns the counts into offsets and the active count
    if (last_block(done)) block_scan256(block_counts, (int)gridDim.x, total);
}

// Reinitialisation list of the local scheme: the entries of the active list
// whose tile holds a point of N (nflag, written by the advance pass).  Tiles
// without N points do not change during the step's reinitialisation
// passes, and both ping-pong buffers already hold their values after the
// advance, so those passes skip them.
__global__ void __launch_bounds__(256) k_nflag_count(const uint8_t* __restrict__ nflag,
                                                     const int* __restrict__ count,
                                                     int* block_counts, unsigned* done,
                                                     int* total)
{
    const int n = *count;
    const int k = blockIdx.x * 256 + threadIdx.x;
    const int on = (k < n) ? (nflag[k] != 0) : 0;
    const int cnt = __syncthreads_count(on);
    if (threadIdx.x == 0) block_counts[blockIdx.x] = cnt;
    if (last_block(done)) block_scan256(block_counts, (int)gridDim.x, total);
}

// ascending compaction of the flagged entries: tile id, info byte and the 64
// bytes of N bits; unflagged entries hold no point of T, so when the tube
// test is due their core flag is 0
__global__ void __launch_bounds__(256) k_nflag_scatter(
    const uint8_t* __restrict__ nflag, const int* __restrict__ count,
    const int* __restrict__ offsets, const int* __restrict__ list,
    const uint8_t* __restrict__ list_info, const uint4* __restrict__ nmask, int* nl,
    uint8_t* nl_info, uint4* nl_mask, uint8_t* core)
{
    __shared__ int warp_cnt[8];
    const int n = *count;
    const int k = blockIdx.x * 256 + threadIdx.x;
    const int on = (k < n) ? (nflag[k] != 0) : 0;
    const unsigned b = __ballot_sync(0xffffffffu, on);
    const int w = threadIdx.x >> 5;
    if (lane_id() == 0) warp_cnt[w] = __popc(b);
    __syncthreads();
    int before = 0;
    for (int i = 0; i < w; ++i) before += warp_cnt[i];
    if (on) {
        const int pos = offsets[blockIdx.x] + before + __popc(b & ((1u << lane_id()) - 1u));
        nl[pos] = list[k];
        nl_info[pos] = list_info[k];
#pragma unroll
        for (int q = 0; q < 4; ++q) nl_mask[(size_t)pos * 4 + q] = nmask[(size_t)k * 4 + q];
    } else if (k < n && core) {
        core[list[k]] = 0;
    }
}

// exclusive scan of up to 1024*32 block counts by one 1024-thread block
__global__ void __launch_bounds__(1024) k_scan(int* counts, int n, int* total)
{
    __shared__ int warp_sums[32];
    const int per = (n + 1023) / 1024;
    const int b0 = threadIdx.x * per;
    int local = 0;
    for (int k = 0; k < per; ++k)
        if (b0 + k < n) local += counts[b0 + k];
    // inclusive warp scan
    int v = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if ((int)lane_id() >= o) v += u;
    }
    if (lane_id() == 31) warp_sums[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        int w = warp_sums[threadIdx.x];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, w, o);
            if ((int)threadIdx.x >= o) w += u;
        }
        warp_sums[threadIdx.x] = w;  // inclusive over warps
    }
    __syncthreads();
    int run = v - local + ((threadIdx.x >> 5) ? warp_sums[(threadIdx.x >> 5) - 1] : 0);
    for (int k = 0; k < per; ++k) {
        if (b0 + k < n) {
            const int c = counts[b0 + k];
            counts[b0 + k] = run;
            run += c;
        }
    }
    if (threadIdx.x == 1023) *total = run;
}

// dt of instance i (Eq. 3 has no rule; CFL: dt = value * h / M, value * h
// when M = 0).  finalize: M from the max|F| bits of the rebuild (or |Fc| for a
// constant speed; 0 for an empty band), bits cleared for the next rebuild.
__device__ void set_dt_one(StepScalars* sc, int i, const Inst& in, int mode, double value,
                           int finalize, int prec, unsigned long long* Mbits, long long n)
{
    double M;
    if (finalize) {
        if (in.speed_mode == 1) {
            M = (n > 0) ? fabs(in.Fc) : 0.0;
        } else {
            const unsigned long long b = __ldcg(Mbits + i);
            M = prec == 0 ? (double)__uint_as_float((unsigned)b) : __longlong_as_double((long long)b);
            if (n == 0) M = 0.0;
        }
        Mbits[i] = 0;
        sc[i].M = M;
    } else {
        M = sc[i].M;
    }
    double dt;
    if (mode == 1) {
        const double ch = __dmul_rn(value, in.h);
        dt = (M > 0.0) ? __ddiv_rn(ch, M) : ch;
    } else {
        dt = value;
    }
    sc[i].dt = dt;
    sc[i].coef = __double2float_rn(__ddiv_rn(dt, in.h));
    sc[i].Fc = __double2float_rn(in.Fc);
}

template <typename T>
__device__ __forceinline__ unsigned long long ordered_bits(T v)
{
    if constexpr (sizeof(T) == 4) return (unsigned long long)__float_as_uint(v);
    else return (unsigned long long)__double_as_longlong(v);
}

// scatter active ids in ascending order; block max of tile max|F| over the
// active tiles -> atomicMax on the ordered bits (values are >= 0).  Tiles
// leaving the active set get their current values copied into the other
// ping-pong buffer (the whole block copies them together), so both buffers
// agree on every inactive tile.
// xface_mode (FP32 single grid; the steps read the x-faces of frozen x
// neighbours from a compact copy, see StepArgs::xface): 0 off; 1 every
// entry's frozen x-faces get their fill bit in list_nact (NACT_FILL_XM /
// _XP: the next filling step reads them in place and writes the copy);
// 2 the copies of the previous band are complete and no value has changed
// since other than by the steps, so only faces whose tile was not active
// before or whose neighbour was (bit 1 of act: active at the previous
// rebuild) get the bit -- a frozen tile keeps its values while it stays
// frozen.
template <typename T>
__global__ void __launch_bounds__(256) k_scatter(const uint8_t* __restrict__ act,
                                                 const int* __restrict__ offsets, int* list,
                                                 uint8_t* list_info,
                                                 const uint8_t* __restrict__ tile_sgn,
                                                 unsigned const_sgn, Inst single,
                                                 long long ntiles, const T* __restrict__ tile_maxF,
                                                 unsigned long long* Mbits,
                                                 const uint4* __restrict__ cur, uint4* other,
                                                 uint8_t* list_nact, StepScalars* sc, int dt_mode,
                                                 double dt_value, const int* count,
                                                 unsigned* done, int xface_mode)
{
    __shared__ int warp_cnt[8];
    __shared__ int warp_leave[8];
    __shared__ unsigned long long warp_max_bits[8];
    __shared__ int leave_ids[256];
    pdl_wait();
    const long long t = (long long)blockIdx.x * 256 + threadIdx.x;
    const bool inb = t < ntiles;
    // every load this thread may need is issued here, independently of the
    // tile's own flag (one round trip instead of a chain of three): the
    // block's offset, the flags of the face neighbours, max|F| and the sign
    const int blk_off = offsets[blockIdx.x];
    const unsigned nb = inb ? nb_bits(t, single) : 0u;
    const long long tpl = (long long)single.tnx * single.tny;
    unsigned nf[6] = {0u, 0u, 0u, 0u, 0u, 0u};  // act of the -x, +x, -y, +y, -z, +z neighbours
    if (list_nact) {
        if (nb & NB_XM) nf[0] = act[t - 1];
        if (nb & NB_XP) nf[1] = act[t + 1];
        if (nb & NB_YM) nf[2] = act[t - single.tnx];
        if (nb & NB_YP) nf[3] = act[t + single.tnx];
        if (nb & NB_ZM) nf[4] = act[t - tpl];
        if (nb & NB_ZP) nf[5] = act[t + tpl];
    }
    const T maxF = (inb && tile_maxF) ? tile_maxF[t] : T(0);
    const unsigned sgn = (inb && tile_sgn) ? (unsigned)tile_sgn[t] : const_sgn;
    const int fl = inb ? act[t] : 0;
    const int on = fl & 1;
    const int leaving = (fl & 2) && !on;
    const unsigned b = __ballot_sync(0xffffffffu, on);
    const unsigned bl = __ballot_sync(0xffffffffu, leaving);
    const int w = threadIdx.x >> 5;
    unsigned long long mb = 0;
    if (on && tile_maxF) mb = ordered_bits(maxF);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, mb, o);
        mb = u > mb ? u : mb;
    }
    if (lane_id() == 0) {
        warp_cnt[w] = __popc(b);
        warp_leave[w] = __popc(bl);
        warp_max_bits[w] = mb;
    }
    __syncthreads();
    int before = 0, lbefore = 0, ltotal = 0;
    for (int k = 0; k < 8; ++k) {
        if (k < w) {
            before += warp_cnt[k];
            lbefore += warp_leave[k];
        }
        ltotal += warp_leave[k];
    }
    const unsigned below = (1u << lane_id()) - 1u;
    if (on) {
        const int pos = blk_off + before + __popc(b & below);
        list[pos] = (int)t;
        list_info[pos] = (uint8_t)(nb | sgn);
        if (list_nact) {
            // the face neighbours inside the domain that are active
            unsigned an = 0u;
#pragma unroll
            for (int k = 0; k < 6; ++k)
                if (nf[k] & 1u) an |= 1u << k;  // NB_XM, NB_XP, NB_YM, NB_YP, NB_ZM, NB_ZP
            const unsigned fz = nb & ~an;
            const bool was = xface_mode == 2 && (fl & 2);
            if (xface_mode && (fz & NB_XM) && !(was && !(nf[0] & 2u))) an |= NACT_FILL_XM;
            if (xface_mode && (fz & NB_XP) && !(was && !(nf[1] & 2u))) an |= NACT_FILL_XP;
            list_nact[pos] = (uint8_t)an;
        }
    }
    if (leaving) leave_ids[lbefore + __popc(bl & below)] = (int)t;
    if (threadIdx.x == 0 && tile_maxF) {
        unsigned long long m = 0;
        for (int k = 0; k < 8; ++k) m = warp_max_bits[k] > m ? warp_max_bits[k] : m;
        if (m) atomicMax(Mbits, m);
    }
    if (ltotal > 0) {
        __syncthreads();
        constexpr int VEC = TILE_PTS * sizeof(T) / 16;  // uint4 per tile
        const int total = ltotal * VEC;
        for (int i = threadIdx.x; i < total; i += 256) {
            const size_t off = (size_t)leave_ids[i / VEC] * VEC + (i % VEC);
            other[off] = cur[off];
        }
    }
    // the last block has every block's max|F| bits: the step's dt
    if (last_block(done) && threadIdx.x == 0)
        set_dt_one(sc, 0, single, dt_mode, dt_value, 1, sizeof(T) == 4 ? 0 : 1, Mbits,
                   (long long)__ldcg(count));
}

// scatter for a batch of instances (FP32): as k_scatter, plus the instance
// id of every entry, per-instance active counts and per-instance max |F|.
// Lanes of a warp usually share an instance; each group of equal instance
// ids folds its count / max with one atomic.
__global__ void __launch_bounds__(256) k_scatter_batch(
    const uint8_t* __restrict__ act, const int* __restrict__ offsets, int* list,
    uint8_t* list_info, uint16_t* list_inst, const uint8_t* __restrict__ tile_sgn,
    const Inst* __restrict__ d_inst, const uint16_t* __restrict__ tile_inst, long long ntiles,
    const float* __restrict__ tile_maxF, unsigned long long* Mbits, int* inst_count,
    const uint4* __restrict__ cur, uint4* other)
{
    __shared__ int warp_cnt[8];
    __shared__ int warp_leave[8];
    __shared__ int leave_ids[256];
    pdl_wait();
    const long long t = (long long)blockIdx.x * 256 + threadIdx.x;
    const int fl = (t < ntiles) ? act[t] : 0;
    const int on = fl & 1;
    const int leaving = (fl & 2) && !on;
    const unsigned b = __ballot_sync(0xffffffffu, on);
    const unsigned bl = __ballot_sync(0xffffffffu, leaving);
    const int w = threadIdx.x >> 5;
    const unsigned inst = (t < ntiles) ? tile_inst[t] : 0xffffu;
    if (lane_id() == 0) {
        warp_cnt[w] = __popc(b);
        warp_leave[w] = __popc(bl);
    }
    // per-instance count and max|F| of the active lanes
    const unsigned key = on ? inst : 0x10000u + lane_id();
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    const unsigned mbits = (on && tile_maxF) ? __float_as_uint(tile_maxF[t]) : 0u;
    const unsigned gmax = __reduce_max_sync(grp, mbits);
    if (on && (__ffs(grp) - 1) == (int)lane_id()) {
        atomicAdd(&inst_count[inst], __popc(grp));
        if (tile_maxF && gmax) atomicMax(&Mbits[inst], (unsigned long long)gmax);
    }
    __syncthreads();
    int before = 0, lbefore = 0, ltotal = 0;
    for (int k = 0; k < 8; ++k) {
        if (k < w) {
            before += warp_cnt[k];
            lbefore += warp_leave[k];
        }
        ltotal += warp_leave[k];
    }
    const unsigned below = (1u << lane_id()) - 1u;
    if (on) {
        const int pos = offsets[blockIdx.x] + before + __popc(b & below);
        const Inst& in = d_inst[inst];
        const unsigned sg = tile_sgn ? tile_sgn[t] : (in.Fc >= 0.0 ? SG_POS : SG_NEG);
        list[pos] = (int)t;
        list_info[pos] = (uint8_t)(nb_bits(t, in) | sg);
        list_inst[pos] = (uint16_t)inst;
    }
    if (leaving) leave_ids[lbefore + __popc(bl & below)] = (int)t;
    if (ltotal == 0) return;
    __syncthreads();
    constexpr int VEC = TILE_PTS * 4 / 16;
    const int total = ltotal * VEC;
    for (int i = threadIdx.x; i < total; i += 256) {
        const size_t off = (size_t)leave_ids[i / VEC] * VEC + (i % VEC);
        other[off] = cur[off];
    }
}

// ---------------------------------------------------------------------------
// Incremental rebuild.  When the steps since the previous rebuild
// ran the fused tube test, core is fresh on every entry of the list and 0 on
// every other tile (a tile whose core flag is set is active), so the new
// active set -- the one-tile dilation of core (Eq. 11 cover) -- is marked
// from the core entries of the previous list alone, and only the
// compaction walks every tile, 16 flag bytes per thread:
//   k_mark           marks[t] = 1 for the neighbourhood of each core entry
//   k_mark_count     per-block counts of the marks, scanned by the last block
//   k_mark_scatter   the ascending list ids, act = new | old << 1, marks
//                    cleared, the ids of the tiles leaving the set
//   k_entry_batch    per entry: info byte, instance, per-instance count and
//                    max |F|; the leaving tiles' copies (then k_set_dt_batch
//                    as after the full scatter)
//   k_entry_single   single grid: per entry the info byte, the active /
//                    frozen-face byte, max |F|; the leaving tiles' copies;
//                    dt in the last block (as k_scatter)
// The list, act, the counts and dt equal those of k_dilate + k_scatter /
// k_scatter_batch.

// 1 for each byte (0..15) of v whose bit 0 is set, packed into bits 0..15
__device__ __forceinline__ unsigned byte_bits16(const uint4& v)
{
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
    unsigned r = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        unsigned x = w[k] & 0x01010101u;   // bits 0, 8, 16, 24
        x |= x >> 7;                       // bytes 0, 1 -> bits 0, 1; bytes 2, 3 -> bits 16, 17
        x = (x | (x >> 14)) & 0xFu;        // bits 16, 17 -> bits 2, 3
        r |= x << (4 * k);
    }
    return r;
}

__global__ void __launch_bounds__(256) k_mark(const int* __restrict__ list,
                                              const int* __restrict__ count,
                                              const uint8_t* __restrict__ core, uint8_t* mark,
                                              const Inst* __restrict__ d_inst,
                                              const uint16_t* __restrict__ tile_inst, Inst single,
                                              int conn)
{
    pdl_wait();
    const int n = *count;
    const bool all26 = conn != 6;
    for (int k = blockIdx.x * 256 + threadIdx.x; k < n; k += gridDim.x * 256) {
        const int t = __ldg(list + k);
        if (!__ldg(core + t)) continue;
        const Inst& in = tile_inst ? d_inst[__ldg(tile_inst + t)] : single;
        const int loc = (int)(t - in.tile_base);
        const int tpl = in.tnx * in.tny;
        const int tz = loc / tpl;
        const int rem = loc - tz * tpl;
        const int ty = rem / in.tnx, tx = rem - ty * in.tnx;
        const bool ex[3] = {tx > 0, true, tx < in.tnx - 1};
        const bool ey[3] = {ty > 0, true, ty < in.tny - 1};
        const bool ez[3] = {tz > 0, true, tz < in.tnz - 1};
        uint8_t* mt = mark + t;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                uint8_t* row = mt + (long long)dz * tpl + (long long)dy * in.tnx;
                const bool vzy = ez[dz + 1] && ey[dy + 1];
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const bool face = abs(dx) + abs(dy) + abs(dz) <= 1;
                    if (vzy && ex[dx + 1] && (face || all26)) row[dx] = 1;
                }
            }
        }
    }
}

// one thread per 16 tiles (nchunks = ceil(ntiles / 16); the flag arrays are
// padded with zero bytes to whole chunks)
__global__ void __launch_bounds__(256) k_mark_count(const uint4* __restrict__ mark, long long nchunks,
                                                    int* block_counts, unsigned* done, int* total,
                                                    int* nleave)
{
    __shared__ int warp_cnt[8];
    pdl_wait();
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    if (i == 0) *nleave = 0;
    int cnt = 0;
    if (i < nchunks) cnt = __popc(byte_bits16(mark[i]));
    const int ws = __reduce_add_sync(0xffffffffu, cnt);
    if (lane_id() == 0) warp_cnt[threadIdx.x >> 5] = ws;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int k = 0; k < 8; ++k) s += warp_cnt[k];
        block_counts[blockIdx.x] = s;
    }
    if (last_block(done)) block_scan256(block_counts, (int)gridDim.x, total);
}

// exclusive prefix over the block of v (each thread's value <= 16), and the
// block's total
__device__ __forceinline__ int block_excl256(int v, int* warp_tot, int& total)
{
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if ((int)lane_id() >= o) inc += u;
    }
    if (lane_id() == 31) warp_tot[threadIdx.x >> 5] = inc;
    __syncthreads();
    int before = 0;
    total = 0;
    for (int k = 0; k < 8; ++k) {
        if (k < (int)(threadIdx.x >> 5)) before += warp_tot[k];
        total += warp_tot[k];
    }
    return before + inc - v;
}

__global__ void __launch_bounds__(256) k_mark_scatter(uint4* mark, uint4* act, long long nchunks,
                                                      const int* __restrict__ offsets, int* list,
                                                      int* leave, int* nleave)
{
    __shared__ int warp_a[8];
    __shared__ int warp_b[8];
    __shared__ int leave_base;
    pdl_wait();
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    uint4 m = make_uint4(0u, 0u, 0u, 0u), a = m;
    if (i < nchunks) {
        m = mark[i];
        a = act[i];
    }
    const unsigned nw = byte_bits16(m);            // active after this rebuild
    const unsigned ol = byte_bits16(a);            // active before it
    const unsigned lv = ol & ~nw;                  // leaving the set
    int ltotal = 0, dummy = 0;
    int pos = block_excl256(__popc(nw), warp_a, dummy) + offsets[blockIdx.x];
    int lpos = block_excl256(__popc(lv), warp_b, ltotal);
    const int t0 = (int)(i * 16);
    for (unsigned b = nw; b; b &= b - 1u) list[pos++] = t0 + __ffs(b) - 1;
    if (i < nchunks) {
        const uint4 o = make_uint4(m.x | ((a.x & 0x01010101u) << 1), m.y | ((a.y & 0x01010101u) << 1),
                                   m.z | ((a.z & 0x01010101u) << 1), m.w | ((a.w & 0x01010101u) << 1));
        act[i] = o;
        mark[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    // the leaving tiles (in any order): copied by the whole next grid, a
    // block holds too many of them to copy them itself
    if (ltotal == 0) return;
    if (threadIdx.x == 0) leave_base = atomicAdd(nleave, ltotal);
    __syncthreads();
    lpos += leave_base;
    for (unsigned b = lv; b; b &= b - 1u) leave[lpos++] = t0 + __ffs(b) - 1;
}

// per list entry (ascending): the info byte and instance of the entry, the
// per-instance active counts and max |F| (as k_scatter_batch)
__global__ void __launch_bounds__(256) k_entry_batch(const int* __restrict__ list,
                                                     const int* __restrict__ count,
                                                     uint8_t* list_info, uint16_t* list_inst,
                                                     const uint8_t* __restrict__ tile_sgn,
                                                     const Inst* __restrict__ d_inst,
                                                     const uint16_t* __restrict__ tile_inst,
                                                     const float* __restrict__ tile_maxF,
                                                     unsigned long long* Mbits, int* inst_count,
                                                     const int* __restrict__ leave,
                                                     const int* __restrict__ nleave,
                                                     const uint4* __restrict__ cur,
                                                     uint4* __restrict__ other)
{
    pdl_wait();
    const int n = *count;
    // the tiles leaving the active set keep their values in both buffers:
    // 128 16-byte words per tile, four independent copies in flight per thread
    {
        constexpr int VEC = TILE_PTS * 4 / 16;
        const long long total = (long long)*nleave * VEC;
        const long long nthr = (long long)gridDim.x * 256;
        for (long long j = (long long)blockIdx.x * 256 + threadIdx.x; j < total; j += 4 * nthr) {
            uint4 v[4];
            size_t off[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long jj = j + u * nthr;
                off[u] = jj < total ? (size_t)__ldg(leave + jj / VEC) * VEC + (size_t)(jj % VEC) : 0;
                if (jj < total) v[u] = cur[off[u]];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (j + u * nthr < total) other[off[u]] = v[u];
        }
    }
    // every thread of a block runs the same number of rounds (warp-wide
    // match / reduce below)
    for (int base = blockIdx.x * 256; base < n; base += gridDim.x * 256) {
        const int k = base + threadIdx.x;
        const bool on = k < n;
        const int t = on ? list[k] : 0;
        const unsigned inst = on ? (unsigned)__ldg(tile_inst + t) : 0xffffu;
        const unsigned key = on ? inst : 0x10000u + lane_id();
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        const unsigned mbits = (on && tile_maxF) ? __float_as_uint(__ldg(tile_maxF + t)) : 0u;
        const unsigned gmax = __reduce_max_sync(grp, mbits);
        if (on && (__ffs(grp) - 1) == (int)lane_id()) {
            atomicAdd(&inst_count[inst], __popc(grp));
            if (tile_maxF && gmax) atomicMax(&Mbits[inst], (unsigned long long)gmax);
        }
        if (on) {
            const Inst& in = d_inst[inst];
            const unsigned sg = tile_sgn ? tile_sgn[t] : (in.Fc >= 0.0 ? SG_POS : SG_NEG);
            list_info[k] = (uint8_t)(nb_bits(t, in) | sg);
            list_inst[k] = (uint16_t)inst;
        }
    }
}

// copies of the leaving tiles (ids in leave[0 .. *nleave)) from cur into
// other, spread over the whole grid: four independent 16-byte copies in
// flight per thread
template <int VEC>
__device__ __forceinline__ void copy_leaving(const int* __restrict__ leave, const int* __restrict__ nleave,
                                             const uint4* __restrict__ cur, uint4* __restrict__ other)
{
    const long long total = (long long)*nleave * VEC;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < total; j += 4 * nthr) {
        uint4 v[4];
        size_t off[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long jj = j + u * nthr;
            off[u] = jj < total ? (size_t)__ldg(leave + jj / VEC) * VEC + (size_t)(jj % VEC) : 0;
            if (jj < total) v[u] = cur[off[u]];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (j + u * nthr < total) other[off[u]] = v[u];
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_entry_single(
    const int* __restrict__ list, const int* __restrict__ count, uint8_t* list_info,
    const uint8_t* __restrict__ act, const uint8_t* __restrict__ tile_sgn, unsigned const_sgn,
    Inst single, const T* __restrict__ tile_maxF, unsigned long long* Mbits, uint8_t* list_nact,
    int xface_mode, const int* __restrict__ leave, const int* __restrict__ nleave,
    const uint4* __restrict__ cur, uint4* __restrict__ other, StepScalars* sc, int dt_mode,
    double dt_value, unsigned* done)
{
    __shared__ unsigned long long warp_max[8];
    pdl_wait();
    const int n = *count;
    copy_leaving<TILE_PTS * (int)sizeof(T) / 16>(leave, nleave, cur, other);
    const long long tpl = (long long)single.tnx * single.tny;
    unsigned long long mb = 0;
    for (int k = blockIdx.x * 256 + threadIdx.x; k < n; k += gridDim.x * 256) {
        const int t = list[k];
        const unsigned nb = nb_bits(t, single);
        const unsigned sgn = tile_sgn ? (unsigned)tile_sgn[t] : const_sgn;
        if (tile_maxF) {
            const unsigned long long u = ordered_bits(tile_maxF[t]);
            mb = u > mb ? u : mb;
        }
        list_info[k] = (uint8_t)(nb | sgn);
        if (list_nact) {
            // act: bit 0 active now, bit 1 active before this rebuild
            unsigned nf[6] = {0u, 0u, 0u, 0u, 0u, 0u};
            if (nb & NB_XM) nf[0] = act[t - 1];
            if (nb & NB_XP) nf[1] = act[t + 1];
            if (nb & NB_YM) nf[2] = act[t - single.tnx];
            if (nb & NB_YP) nf[3] = act[t + single.tnx];
            if (nb & NB_ZM) nf[4] = act[t - tpl];
            if (nb & NB_ZP) nf[5] = act[t + tpl];
            const unsigned fl = act[t];
            unsigned an = 0u;
#pragma unroll
            for (int q = 0; q < 6; ++q)
                if (nf[q] & 1u) an |= 1u << q;  // NB_XM, NB_XP, NB_YM, NB_YP, NB_ZM, NB_ZP
            const unsigned fz = nb & ~an;
            const bool was = xface_mode == 2 && (fl & 2u);
            if (xface_mode && (fz & NB_XM) && !(was && !(nf[0] & 2u))) an |= NACT_FILL_XM;
            if (xface_mode && (fz & NB_XP) && !(was && !(nf[1] & 2u))) an |= NACT_FILL_XP;
            list_nact[k] = (uint8_t)an;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, mb, o);
        mb = u > mb ? u : mb;
    }
    if (lane_id() == 0) warp_max[threadIdx.x >> 5] = mb;
    __syncthreads();
    if (threadIdx.x == 0 && tile_maxF) {
        unsigned long long m = 0;
        for (int q = 0; q < 8; ++q) m = warp_max[q] > m ? warp_max[q] : m;
        if (m) atomicMax(Mbits, m);
    }
    // the last block has every block's max |F| bits: the step's dt
    if (last_block(done) && threadIdx.x == 0)
        set_dt_one(sc, 0, single, dt_mode, dt_value, 1, sizeof(T) == 4 ? 0 : 1, Mbits,
                   (long long)__ldcg(count));
}

// per-instance dt (one thread per instance)
__global__ void k_set_dt_batch(StepScalars* sc, int n_inst, const Inst* __restrict__ d_inst,
                               int mode, double value, int finalize, unsigned long long* Mbits,
                               int* inst_count)
{
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inst) return;
    const Inst& in = d_inst[i];
    double M;
    if (finalize) {
        const int n = inst_count[i];
        if (in.speed_mode == 1) M = (n > 0) ? fabs(in.Fc) : 0.0;
        else M = (n > 0) ? (double)__uint_as_float((unsigned)Mbits[i]) : 0.0;
        Mbits[i] = 0;
        inst_count[i] = 0;
        sc[i].M = M;
        sc[i].active = n;
    } else {
        M = sc[i].M;
    }
    double dt;
    if (mode == 1) {
        const double ch = __dmul_rn(value, in.h);
        dt = (M > 0.0) ? __ddiv_rn(ch, M) : ch;
    } else {
        dt = value;
    }
    sc[i].dt = dt;
    sc[i].coef = __double2float_rn(__ddiv_rn(dt, in.h));
    sc[i].Fc = __double2float_rn(in.Fc);
}

// full-domain list: every tile in ascending order
__global__ void __launch_bounds__(256) k_full_list(int* list, uint8_t* list_info,
                                                   const uint8_t* __restrict__ tile_sgn,
                                                   unsigned const_sgn, Inst single,
                                                   long long ntiles, int* count,
                                                   uint8_t* list_nact)
{
    for (long long t = (long long)blockIdx.x * 256 + threadIdx.x; t < ntiles;
         t += (long long)gridDim.x * 256) {
        list[t] = (int)t;
        const unsigned nb = nb_bits(t, single);
        list_info[t] = (uint8_t)(nb | (tile_sgn ? tile_sgn[t] : const_sgn));
        if (list_nact) list_nact[t] = (uint8_t)nb;  // every tile is active
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = (int)ntiles;
}

// max of tile max|F| over all tiles (full-domain CFL bound)
template <typename T>
__global__ void __launch_bounds__(256) k_max_all(const T* __restrict__ tile_maxF, long long ntiles,
                                                 unsigned long long* Mbits)
{
    unsigned long long mb = 0;
    for (long long t = (long long)blockIdx.x * 256 + threadIdx.x; t < ntiles;
         t += (long long)gridDim.x * 256) {
        const unsigned long long u = ordered_bits(tile_maxF[t]);
        mb = u > mb ? u : mb;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, mb, o);
        mb = u > mb ? u : mb;
    }
    if (lane_id() == 0 && mb) atomicMax(Mbits, mb);
}

// dt from M, FP64, single thread per instance.  finalize: M comes from the
// reduction bits (then cleared); otherwise the stored M is reused.
__global__ void k_set_dt(StepScalars* sc, int n_inst, const Inst* d_inst, Inst single, int mode,
                         double value, int finalize, int prec, unsigned long long* Mbits,
                         const int* count, long long fixed_count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inst) return;
    const Inst& in = d_inst ? d_inst[i] : single;
    const long long n = count ? (long long)*count : fixed_count;
    set_dt_one(sc, i, in, mode, value, finalize, prec, Mbits, n);
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int conv_grid(long long ntiles)
{
    const long long g = ntiles < (1 << 20) ? ntiles : (1 << 20);
    return (int)(g > 0 ? g : 1);
}

cudaError_t launch_pack(const void* src, void* dst, const Inst& in, int prec, unsigned* nonfinite,
                        cudaStream_t s)
{
    if (prec == 0)
        k_convert<float, true><<<conv_grid(in.ntiles), 128, 0, s>>>(
            (const float*)src, (float*)dst, in, nonfinite);
    else
        k_convert<double, true><<<conv_grid(in.ntiles), 128, 0, s>>>(
            (const double*)src, (double*)dst, in, nonfinite);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_copy16(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                uint4* __restrict__ dst2, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (size_t)gridDim.x * 256) {
        const uint4 v = src[i];
        dst[i] = v;
        if (dst2) dst2[i] = v;
    }
}

cudaError_t launch_copy(void* dst, const void* src, size_t bytes, cudaStream_t s, void* dst2)
{
    const size_t n = bytes / 16;
    if (n == 0) return cudaSuccess;
    size_t g = (n + 255) / 256;
    if (g > 148 * 16) g = 148 * 16;
    k_copy16<<<(int)g, 256, 0, s>>>((const uint4*)src, (uint4*)dst, (uint4*)dst2, n);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const void* src, void* dst, const Inst& in, int prec, cudaStream_t s)
{
    if (prec == 0)
        k_convert<float, false><<<conv_grid(in.ntiles), 128, 0, s>>>(
            (const float*)src, (float*)dst, in, nullptr);
    else
        k_convert<double, false><<<conv_grid(in.ntiles), 128, 0, s>>>(
            (const double*)src, (double*)dst, in, nullptr);
    return cudaGetLastError();
}

static int warp_grid(long long ntiles)
{
    long long g = (ntiles + 7) / 8;
    if (g > 148 * 64) g = 148 * 64;
    return (int)(g > 0 ? g : 1);
}

cudaError_t launch_tile_speed(const void* F, void* tile_maxF, uint8_t* tile_sgn, long long ntiles,
                              int prec, cudaStream_t s)
{
    if (prec == 0)
        k_tile_speed<float><<<warp_grid(ntiles), 256, 0, s>>>((const float*)F, (float*)tile_maxF,
                                                              tile_sgn, ntiles);
    else
        k_tile_speed<double><<<warp_grid(ntiles), 256, 0, s>>>((const double*)F,
                                                               (double*)tile_maxF, tile_sgn, ntiles);
    return cudaGetLastError();
}

cudaError_t launch_classify_all(const void* phi, uint8_t* core, const Inst* d_inst,
                                const uint16_t* tile_inst, const Inst& single, long long ntiles,
                                int prec, cudaStream_t s)
{
    if (prec == 0)
        k_classify_all<float><<<warp_grid(ntiles), 256, 0, s>>>((const float*)phi, core, d_inst,
                                                                tile_inst, single, ntiles);
    else
        k_classify_all<double><<<warp_grid(ntiles), 256, 0, s>>>((const double*)phi, core, d_inst,
                                                                 tile_inst, single, ntiles);
    return cudaGetLastError();
}

__global__ void k_row_counts(const int* __restrict__ list, const int* __restrict__ count,
                             int tiles_per_row, int* rows, int capacity)
{
    const int n = *count;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int r = list[k] / tiles_per_row;
        if (r < capacity) atomicAdd(&rows[r], 1);
    }
}

// dt from an external bound: M = *Mext (e.g. the maximum over the slabs of
// a split grid), dt = cfl h / M (cfl h when M = 0), as at a rebuild
__global__ void k_set_dt_from(StepScalars* sc, const double* Mext, Inst single, double cfl, int prec)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    sc[0].M = *Mext;
    set_dt_one(sc, 0, single, 1, cfl, 0, prec, nullptr, 0);
}

cudaError_t launch_set_dt_from(StepScalars* sc, const double* Mext, const Inst& in, double cfl,
                               int prec, cudaStream_t s)
{
    k_set_dt_from<<<1, 32, 0, s>>>(sc, Mext, in, cfl, prec);
    return cudaGetLastError();
}

// chunk copy: chunk t of `words` 32-bit words from src + t * src_stride to
// dst + t * dst_stride (a z-plane of each tile of a tile row, between the
// bricked layout and a packed buffer or another context's ghost row)
__global__ void k_chunk_copy(const uint32_t* __restrict__ src, long long src_stride,
                             uint32_t* __restrict__ dst, long long dst_stride, int words,
                             long long nchunks)
{
    const long long n = nchunks * words;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long t = i / words;
        const int j = (int)(i - t * words);
        dst[t * dst_stride + j] = src[t * src_stride + j];
    }
}

cudaError_t launch_chunk_copy(const void* src, long long src_stride_words, void* dst,
                              long long dst_stride_words, int words, long long nchunks, cudaStream_t s)
{
    const long long n = nchunks * words;
    long long g = (n + 255) / 256;
    if (g > 148 * 8) g = 148 * 8;
    k_chunk_copy<<<(int)(g > 0 ? g : 1), 256, 0, s>>>((const uint32_t*)src, src_stride_words,
                                                       (uint32_t*)dst, dst_stride_words, words, nchunks);
    return cudaGetLastError();
}

cudaError_t launch_row_counts(const int* list, const int* count, int tiles_per_row, int* rows,
                              int capacity, cudaStream_t s)
{
    k_row_counts<<<148, 256, 0, s>>>(list, count, tiles_per_row, rows, capacity);
    return cudaGetLastError();
}

cudaError_t launch_dilate(const uint8_t* core, uint8_t* act, int* block_counts,
                          const Inst* d_inst, const uint16_t* tile_inst, const Inst& single,
                          long long ntiles, unsigned* done, int* count, int conn, cudaStream_t s)
{
    const int nb = (int)((ntiles + 255) / 256);
    return launch_after(k_dilate, nb, 256, s, core, act, block_counts, d_inst, tile_inst, single,
                        ntiles, done, count, conn);
}

cudaError_t launch_nflag_count(const uint8_t* nflag, const int* count, int* block_counts,
                               int nblocks, unsigned* done, int* total, cudaStream_t s)
{
    k_nflag_count<<<nblocks, 256, 0, s>>>(nflag, count, block_counts, done, total);
    return cudaGetLastError();
}

cudaError_t launch_nflag_scatter(const uint8_t* nflag, const int* count, const int* block_offsets,
                                 const int* list, const uint8_t* list_info, const uint32_t* nmask,
                                 int* nl, uint8_t* nl_info, uint32_t* nl_mask, uint8_t* core,
                                 int nblocks, cudaStream_t s)
{
    k_nflag_scatter<<<nblocks, 256, 0, s>>>(nflag, count, block_offsets, list, list_info,
                                            (const uint4*)nmask, nl, nl_info, (uint4*)nl_mask, core);
    return cudaGetLastError();
}

cudaError_t launch_scan(int* block_counts, int nblocks, int* count, cudaStream_t s)
{
    k_scan<<<1, 1024, 0, s>>>(block_counts, nblocks, count);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const uint8_t* act, const int* block_offsets, int* list,
                           uint8_t* list_info, const uint8_t* tile_sgn, unsigned const_sgn,
                           const Inst& single, long long ntiles, const void* tile_maxF, int prec,
                           unsigned long long* Mbits, const void* cur, void* other,
                           uint8_t* list_nact, StepScalars* sc, int dt_mode, double dt_value,
                           const int* count, unsigned* done, int xface_mode, cudaStream_t s)
{
    const int nb = (int)((ntiles + 255) / 256);
    if (prec == 0)
        return launch_after(k_scatter<float>, nb, 256, s, act, block_offsets, list, list_info,
                            tile_sgn, const_sgn, single, ntiles, (const float*)tile_maxF, Mbits,
                            (const uint4*)cur, (uint4*)other, list_nact, sc, dt_mode, dt_value,
                            count, done, xface_mode);
    return launch_after(k_scatter<double>, nb, 256, s, act, block_offsets, list, list_info,
                        tile_sgn, const_sgn, single, ntiles, (const double*)tile_maxF, Mbits,
                        (const uint4*)cur, (uint4*)other, list_nact, sc, dt_mode, dt_value, count,
                        done, 0);
}

cudaError_t launch_scatter_batch(const uint8_t* act, const int* block_offsets, int* list,
                                 uint8_t* list_info, uint16_t* list_inst,
                                 const uint8_t* tile_sgn, const Inst* d_inst,
                                 const uint16_t* tile_inst, long long ntiles,
                                 const void* tile_maxF, int prec, unsigned long long* Mbits,
                                 int* inst_count, const void* cur, void* other, cudaStream_t s)
{
    if (prec != 0) return cudaErrorInvalidValue;
    const int nb = (int)((ntiles + 255) / 256);
    return launch_after(k_scatter_batch, nb, 256, s, act, block_offsets, list, list_info, list_inst,
                        tile_sgn, d_inst, tile_inst, ntiles, (const float*)tile_maxF, Mbits, inst_count,
                        (const uint4*)cur, (uint4*)other);
}

static int band_sm_count()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    return sms;
}

cudaError_t launch_mark(const int* list, const int* count, const uint8_t* core, uint8_t* mark,
                        const Inst* d_inst, const uint16_t* tile_inst, const Inst& single,
                        long long ntiles, int conn, cudaStream_t s)
{
    long long nb = (ntiles + 255) / 256;
    if (nb > 8LL * band_sm_count()) nb = 8LL * band_sm_count();
    return launch_after(k_mark, (int)nb, 256, s, list, count, core, mark, d_inst, tile_inst, single, conn);
}

cudaError_t launch_entry_single(const int* list, const int* count, uint8_t* list_info,
                                const uint8_t* act, const uint8_t* tile_sgn, unsigned const_sgn,
                                const Inst& single, long long ntiles, const void* tile_maxF, int prec,
                                unsigned long long* Mbits, uint8_t* list_nact, int xface_mode,
                                const int* leave, const int* nleave, const void* cur, void* other,
                                StepScalars* sc, int dt_mode, double dt_value, unsigned* done,
                                cudaStream_t s)
{
    long long nb = (ntiles + 255) / 256;
    if (nb > 8LL * band_sm_count()) nb = 8LL * band_sm_count();
    if (prec == 0)
        return launch_after(k_entry_single<float>, (int)nb, 256, s, list, count, list_info, act, tile_sgn,
                            const_sgn, single, (const float*)tile_maxF, Mbits, list_nact, xface_mode,
                            leave, nleave, (const uint4*)cur, (uint4*)other, sc, dt_mode, dt_value, done);
    return launch_after(k_entry_single<double>, (int)nb, 256, s, list, count, list_info, act, tile_sgn,
                        const_sgn, single, (const double*)tile_maxF, Mbits, list_nact, xface_mode,
                        leave, nleave, (const uint4*)cur, (uint4*)other, sc, dt_mode, dt_value, done);
}

int mark_chunk_blocks(long long ntiles) { return (int)((ntiles + 4095) / 4096); }

cudaError_t launch_mark_count(const uint8_t* mark, long long ntiles, int* block_counts,
                              unsigned* done, int* count, int* nleave, cudaStream_t s)
{
    const long long nchunks = (ntiles + 15) / 16;
    return launch_after(k_mark_count, mark_chunk_blocks(ntiles), 256, s, (const uint4*)mark, nchunks,
                        block_counts, done, count, nleave);
}

cudaError_t launch_mark_scatter(uint8_t* mark, uint8_t* act, long long ntiles,
                                const int* block_offsets, int* list, int* leave, int* nleave,
                                cudaStream_t s)
{
    const long long nchunks = (ntiles + 15) / 16;
    return launch_after(k_mark_scatter, mark_chunk_blocks(ntiles), 256, s, (uint4*)mark, (uint4*)act,
                        nchunks, block_offsets, list, leave, nleave);
}

cudaError_t launch_entry_batch(const int* list, const int* count, uint8_t* list_info,
                               uint16_t* list_inst, const uint8_t* tile_sgn, const Inst* d_inst,
                               const uint16_t* tile_inst, long long ntiles, const void* tile_maxF,
                               int prec, unsigned long long* Mbits, int* inst_count,
                               const int* leave, const int* nleave, const void* cur, void* other,
                               cudaStream_t s)
{
    if (prec != 0) return cudaErrorInvalidValue;
    long long nb = (ntiles + 255) / 256;
    if (nb > 8LL * band_sm_count()) nb = 8LL * band_sm_count();
    return launch_after(k_entry_batch, (int)nb, 256, s, list, count, list_info, list_inst, tile_sgn,
                        d_inst, tile_inst, (const float*)tile_maxF, Mbits, inst_count, leave, nleave,
                        (const uint4*)cur, (uint4*)other);
}

cudaError_t launch_set_dt_batch(StepScalars* sc, int n_inst, const Inst* d_inst, int mode,
                                double value, int finalize, int prec, unsigned long long* Mbits,
                                int* inst_count, cudaStream_t s)
{
    (void)prec;
    return launch_after(k_set_dt_batch, (n_inst + 127) / 128, 128, s, sc, n_inst, d_inst, mode, value,
                        finalize, Mbits, inst_count);
}

cudaError_t launch_full_list(int* list, uint8_t* list_info, const uint8_t* tile_sgn,
                             unsigned const_sgn, const Inst& single, long long ntiles, int* count,
                             uint8_t* list_nact, cudaStream_t s)
{
    long long g = (ntiles + 255) / 256;
    if (g > 148 * 16) g = 148 * 16;
    k_full_list<<<(int)(g > 0 ? g : 1), 256, 0, s>>>(list, list_info, tile_sgn, const_sgn, single,
                                                     ntiles, count, list_nact);
    return cudaGetLastError();
}

cudaError_t launch_max_all(const void* tile_maxF, long long ntiles, int prec,
                           unsigned long long* Mbits, cudaStream_t s)
{
    long long g = (ntiles + 255) / 256;
    if (g > 148 * 8) g = 148 * 8;
    if (g < 1) g = 1;
    if (prec == 0)
        k_max_all<float><<<(int)g, 256, 0, s>>>((const float*)tile_maxF, ntiles, Mbits);
    else
        k_max_all<double><<<(int)g, 256, 0, s>>>((const double*)tile_maxF, ntiles, Mbits);
    return cudaGetLastError();
}

cudaError_t launch_set_dt(StepScalars* sc, int n_inst, const Inst* d_inst, const Inst& single,
                          int mode, double value, int finalize, int prec,
                          unsigned long long* Mbits, const int* count, long long fixed_count,
                          cudaStream_t s)
{
    k_set_dt<<<(n_inst + 127) / 128, 128, 0, s>>>(sc, n_inst, d_inst, single, mode, value,
                                                   finalize, prec, Mbits, count, fixed_count);
    return cudaGetLastError();
}

}  // namespace lsk
