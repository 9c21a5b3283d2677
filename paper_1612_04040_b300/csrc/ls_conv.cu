// ls_conv.cu -- 3x3x3 convolution (16 -> 16 channels, zero padding) as an
// implicit GEMM on the 5th-generation tensor cores (tcgen05), for the learned
// coarse-grid corrector.  This part is not in the paper.
//
// Data: activations are BF16, channels-last act[(z*ny + y)*nx + x][16]; the
// GEMM for one output point m and one tap t is  D[m][n] += sum_k
// X[m + off(t)][k] * W[t][k][n]  with K = N = 16 channels, accumulated in FP32
// over the 27 taps.
//
// A block is 8 x 16 x 4 output points (x, y, z): one 8^3 tile wide in x,
// two in y, half a tile in z, so a block list can follow the band's tiles.
// The TMA engine loads the halo'd input block (10 x 18 x 6 points x 16
// channels) as two 4-D boxes (8 channels, x, y, z), one per half of the
// channels (the second tensor map starts 16 bytes into the activations), so
// shared memory holds X_s[half][z][y][x][8]: every run of 8 consecutive
// points x 8 channels is one contiguous 128-byte "core matrix" of the
// canonical no-swizzle K-major operand layout.  An M-tile is 8 x-points x
// 16 y-rows = 128 points of one z-plane of the halo'd block: its 16 groups
// of 8 points are the 16 rows, one 10-point row apart (SBO = 160 B), and
// the A operand of any (dx, dy) shift is just a descriptor whose start
// address is shifted by it (LBO = one channel-half plane): no im2col copy.
// Points outside the grid are zero-filled by the TMA (zero padding for
// free).
//
// The three dz taps share their A operand: for input plane i of the halo'd
// block and shift (dx, dy), one MMA with N = 48 (dz = -1, 0, 1 stacked x 16
// output channels) gives D_i[p][dz, o] = sum_c X_i[p + (dx, dy)][c]
// W[dx, dy, dz][c][o], accumulated over the 9 shifts; output plane j then
// sums D_j[-1], D_{j+1}[0], D_{j+2}[+1] in the epilogue.  That is 9 x 6 = 54
// MMAs per block (the first and last input planes feed one output plane
// and take N = 16) instead of 27 per output plane: the tensor core's
// operand reads (a 4 KB A tile per MMA) bound this layer.  Weights are
// packed once per launch into the B layout.  The epilogue reads TMEM with
// tcgen05.ld (warp w owns lanes 32w..32w+31, i.e. y-rows 4w..4w+3) and
// applies bias + ReLU, bias only (last layer), or the ReLU mask of the
// backward pass.  An optional list of blocks restricts the work (the
// corrected step needs the network only near the band).
//
// Every wait on an mbarrier is bounded; on timeout the kernel records
// ST_TIMEOUT in the status word, stops issuing work, frees its TMEM and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "ls.h"
#include "ls_internal.cuh"
#include "ls_stencil.cuh"

namespace lsk {

namespace {

constexpr int BXP = 8, BYP = 16, BZP = 4;  // output points of a block per axis
constexpr int PX = BXP + 2, PY = BYP + 2, PZ = BZP + 2;
constexpr int PB = PX * PY * PZ;   // points in the halo'd block
constexpr int HALF_BYTES = PB * 16;
constexpr int XS_BYTES = 2 * HALF_BYTES;
constexpr int W_BYTES = 27 * 512;  // 9 shifts x (48 x 16 bf16)
constexpr int W_PAIR = 48 * 16 * 2;  // bytes of one (dx, dy) shift: N = 48 (dz, o), K = 16
constexpr int MT = BZP;            // output z-planes per block
constexpr int A_SBO = PX * 16;     // between the 8-point groups (y-rows) of an M-tile
constexpr long long WAIT_LIMIT = 1ll << 26;

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait for the phase with the given parity; false on timeout: after
// `limit` polls or WAIT_NS nanoseconds, whichever comes first (a poll of
// try_wait may suspend the thread for a while, so the poll count alone can
// take minutes)
constexpr unsigned long long WAIT_NS = 2000000000ull;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                          long long limit = WAIT_LIMIT)
{
    const unsigned a = smem_u32(bar);
    const unsigned long long t0 = global_ns();
    for (long long i = 0; i < limit; ++i) {
        unsigned ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "  selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((i & 255) == 255 && global_ns() - t0 > WAIT_NS) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// shared-memory matrix descriptor, no swizzle (canonical K-major layout):
// start address, leading (K-direction) and stride (M/N-direction) byte
// offsets of the 8-row x 16-byte core matrices
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((addr & 0x3FFFFu) >> 4);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;  // descriptor version for this architecture
    return d;         // base offset 0, swizzle mode 0 (none)
}

// instruction descriptor, kind::f16: D F32, A and B BF16, both K-major,
// M = 128, N = 16 (IDESC) or 48 (IDESC48)
constexpr unsigned IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
constexpr unsigned IDESC48 = (1u << 4) | (1u << 7) | (1u << 10) | ((48u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_bf16(unsigned d_tmem, unsigned long long a, unsigned long long b,
                                         unsigned accumulate, unsigned idesc = IDESC)
{
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
        "  tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned long long* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16])
{
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

struct ConvArgs {
    const __nv_bfloat16* wpack;  // packed B operand, 27 x 512 bytes
    const float* bias;           // 16 (fwd modes) or NULL
    const __nv_bfloat16* mask;   // backward mode: forward activation of the input layer
    __nv_bfloat16* out_bf16;     // hidden / backward modes: [p][16]
    float* out_f32;              // last-layer mode: [p] (channel 0)
    unsigned* status;
    const int* blist;            // blocks to compute (NULL: every block)
    const int* bcount;           // their number (device)
    int nx, ny, nz;
    int mode;                    // 0 bias+ReLU, 1 bias (channel 0, FP32), 2 ReLU mask
};

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Warp-specialised pipeline, one CTA per SM, 6 warps:
//   warp 0      TMA producer: halo'd input block -> shared stage s (2 stages)
//   warp 1      TMEM owner and MMA issuer: 6 input planes x 9 shifts into
//               TMEM accumulator buffer b (2 buffers x 256 columns)
//   warps 2..5  epilogue: TMEM -> registers -> global (warp w reads lane
//               quadrant w % 4)
// Barriers: full[s] (TMA bytes landed), empty[s] (MMAs reading stage s
// finished), acc_full[b] (accumulators ready), acc_empty[b] (epilogue done,
// 4 arrivals).  Block i of this CTA uses stage and buffer i % 2.
constexpr int NSTAGE = 3;
constexpr int CONV_THREADS = 192;
constexpr int ACC_COLS = 256;  // per accumulator buffer (224 used)
// TMEM column of input plane i's dz group g: plane 0 holds only g = 0 (its
// only output is plane 0), plane MT + 1 only g = 2, the others all three
__host__ __device__ constexpr int acc_col(int i, int g)
{
    return i == 0 ? 0 : (i == MT + 1 ? 16 + 48 * MT : 16 + 48 * (i - 1) + 16 * g);
}

__global__ void __launch_bounds__(CONV_THREADS, 1) k_conv3_tc(const __grid_constant__ CUtensorMap map0,
                                                              const __grid_constant__ CUtensorMap map1,
                                                              ConvArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* ws = smem + NSTAGE * XS_BYTES;  // packed weights
    __shared__ __align__(8) unsigned long long full[NSTAGE], empty[NSTAGE], acc_full[2], acc_empty[2];
    __shared__ unsigned tmem_base_s;
    __shared__ volatile int abort_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int i = tid; i < W_BYTES / 16; i += CONV_THREADS)
        reinterpret_cast<uint4*>(ws)[i] = reinterpret_cast<const uint4*>(a.wpack)[i];
    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);
        }
        abort_s = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_s)),
                     "r"(2 * ACC_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = tmem_base_s;
    const int nbx = a.nx / BXP, nby = a.ny / BYP;
    const int nblocks = a.bcount ? *a.bcount : nbx * nby * (a.nz / BZP);
    const unsigned xs_addr = smem_u32(smem), ws_addr = smem_u32(ws);

    if (warp == 0) {
        if (lane == 0) {
            int i = 0;
            for (int k = blockIdx.x; k < nblocks && !abort_s; k += gridDim.x, ++i) {
                const int s = i % NSTAGE, u = i / NSTAGE;
                if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1)) {
                    atomicOr(a.status, ST_TIMEOUT);
                    abort_s = 1;
                    break;
                }
                const int blk = a.blist ? a.blist[k] : k;
                const int bx = blk % nbx, by = (blk / nbx) % nby, bz = blk / (nbx * nby);
                unsigned char* xs = smem + s * XS_BYTES;
                mbar_expect_tx(&full[s], XS_BYTES);
                tma_load_4d(xs, &map0, 0, bx * BXP - 1, by * BYP - 1, bz * BZP - 1, &full[s]);
                tma_load_4d(xs + HALF_BYTES, &map1, 0, bx * BXP - 1, by * BYP - 1, bz * BZP - 1, &full[s]);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int i = 0;
            for (int k = blockIdx.x; k < nblocks && !abort_s; k += gridDim.x, ++i) {
                const int s = i % NSTAGE, u = i / NSTAGE;
                const int b = i % 2, ub = i / 2;
                if (!mbar_wait(&full[s], u & 1) || (ub > 0 && !mbar_wait(&acc_empty[b], (ub - 1) & 1))) {
                    atomicOr(a.status, ST_TIMEOUT);
                    abort_s = 1;
                    break;
                }
                fence_after();
                // descriptors are linear in the start address (field =
                // address >> 4, all shared addresses < 256 KB): the 216 MMAs
                // of a block differ only by compile-time offsets
                const unsigned long long da = smem_desc(xs_addr + s * XS_BYTES, HALF_BYTES, A_SBO);
                const unsigned long long db = smem_desc(ws_addr, W_PAIR / 2, 128);
                const unsigned acc = tmem + b * ACC_COLS;
#pragma unroll
                for (int i = 0; i < MT + 2; ++i) {
#pragma unroll
                    for (int p = 0; p < 9; ++p) {
                        // input plane i, y-row 0 + (dy + 1), x 0 + (dx + 1) of the halo'd block
                        const unsigned long long a_ = da + (unsigned long long)((i * PY + p / 3) * PX + p % 3);
                        const unsigned long long b_ = db + (unsigned long long)(p * (W_PAIR / 16));
                        if (i == 0)
                            mma_bf16(acc + acc_col(0, 0), a_, b_, p > 0 ? 1u : 0u);
                        else if (i == MT + 1)  // the dz = +1 group: 2 x 8 rows of N in
                            mma_bf16(acc + acc_col(i, 2), a_, b_ + 2 * 16, p > 0 ? 1u : 0u);
                        else
                            mma_bf16(acc + acc_col(i, 0), a_, b_, p > 0 ? 1u : 0u, IDESC48);
                    }
                }
                mma_commit(&empty[s]);
                mma_commit(&acc_full[b]);
            }
        }
    } else {
        // epilogue warps: lane quadrant q = warp % 4 -> M rows 32 q + lane,
        // i.e. point (x0 + lane % 8, y0 + 4 q + lane / 8) of every z-plane
        const int q = warp & 3;
        int i = 0;
        for (int k = blockIdx.x; k < nblocks && !abort_s; k += gridDim.x, ++i) {
            const int b = i % 2, ub = i / 2;
            const int blk = a.blist ? a.blist[k] : k;
            const int bx = blk % nbx, by = (blk / nbx) % nby, bz = blk / (nbx * nby);
            const int x = bx * BXP + (lane & 7);
            const int y = by * BYP + 4 * q + (lane >> 3);
            // the backward pass's ReLU mask does not depend on the MMAs: its
            // loads go out before the wait for the accumulators
            uint4 mk[MT][2];
            if (a.mode == 2) {
#pragma unroll
                for (int j = 0; j < MT; ++j) {
                    const size_t pidx = ((size_t)(bz * BZP + j) * a.ny + y) * a.nx + x;
                    const uint4* mp = reinterpret_cast<const uint4*>(a.mask + pidx * 16);
                    mk[j][0] = mp[0];
                    mk[j][1] = mp[1];
                }
            }
            // the lanes agree before the warp-collective TMEM loads
            if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[b], ub & 1) ? 1 : 0)) {
                if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
                abort_s = 1;
                break;
            }
            fence_after();
#pragma unroll
            for (int j = 0; j < MT; ++j) {
                const int z = bz * BZP + j;
                float v[16], v1[16], v2[16];
                const unsigned tb = tmem + b * ACC_COLS + ((unsigned)(32 * q) << 16);
                tmem_ld16(tb + acc_col(j, 0), v);
                tmem_ld16(tb + acc_col(j + 1, 1), v1);
                tmem_ld16(tb + acc_col(j + 2, 2), v2);
#pragma unroll
                for (int c = 0; c < 16; ++c) v[c] = (v[c] + v1[c]) + v2[c];
                const size_t pidx = ((size_t)z * a.ny + y) * a.nx + x;
                if (a.mode == 1) {
                    a.out_f32[pidx] = v[0] + a.bias[0];
                    continue;
                }
                if (a.mode == 0) {
#pragma unroll
                    for (int c = 0; c < 16; ++c) v[c] = fmaxf(v[c] + a.bias[c], 0.f);
                } else {
                    const __nv_bfloat16* mb0 = reinterpret_cast<const __nv_bfloat16*>(&mk[j][0]);
                    const __nv_bfloat16* mb1 = reinterpret_cast<const __nv_bfloat16*>(&mk[j][1]);
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        if (!(__bfloat162float(mb0[c]) > 0.f)) v[c] = 0.f;
                        if (!(__bfloat162float(mb1[c]) > 0.f)) v[8 + c] = 0.f;
                    }
                }
                uint4 o[2];
                __nv_bfloat162* ob = reinterpret_cast<__nv_bfloat162*>(o);
#pragma unroll
                for (int c = 0; c < 8; ++c) ob[c] = __floats2bfloat162_rn(v[2 * c], v[2 * c + 1]);
                uint4* dp = reinterpret_cast<uint4*>(a.out_bf16 + pidx * 16);
                dp[0] = o[0];
                dp[1] = o[1];
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
    }
    // all roles done (or aborted): MMAs issued by warp 1 have completed once
    // the epilogue has consumed every accumulator; on abort, give in-flight
    // work one more bounded wait before releasing TMEM
    fence_before();
    __syncthreads();
    if (abort_s && tid == 32) {
        for (int b = 0; b < 2; ++b) mbar_wait(&acc_full[b], 0, 1 << 20);
    }
    __syncthreads();
    fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(2 * ACC_COLS)
                     : "memory");
}

// ---- weight gradient on the tensor cores --------------------------------
//
// dW[t][c][o] = sum_p x[p + off(t)][c] dy[p][o] and db[o] = sum_p dy[p][o].
// A tap is split as (dx, dy, dz) = (0, dy, dz) + (dx, 0, 0): with
// q = p + (dx, 0, 0),
//   dW[t][c][o] = sum_q x[q + (0, dy, dz)][c] dy[q - (dx, 0, 0)][o],
// one GEMM per CTA with M = ((dy, dz) pair, input channel), N = (dx, output
// channel) = 48 and K = the points q of the CTA's chunks (64 consecutive
// x-points of one (y, z) row each; out-of-grid points zero-filled by the
// TMA, which is the convolution's zero padding on both operands).  Both
// operands are MN-major (the 8 channels of a point are one contiguous
// 16-byte run).  Per chunk the TMA loads, per dz and channel half, one box
// of x holding the three rows y - 1, y, y + 1 (3 KB), the boxes in the
// order (dz, half), so the 18 8-channel groups of the (dy, dz) pairs sit at
// one stride (SBO = 1 KB) in the order (dz, half, dy); and 3 boxes of dy per
// half (one per dx, 1 KB) for the N operand.  The 8-point groups sit at
// 128 B (LBO).  M-tile 0 holds groups 0..15, M-tile 1 groups 16, 17 and two
// groups of ones kept in shared memory, whose rows accumulate
// sum_q dy[q][o] (the bias gradient, from the dx = 0 columns); the rest of
// M-tile 1 repeats them and is discarded.  The 96-column accumulator lives
// in TMEM across all of a CTA's chunks; the epilogue adds it to dW and db
// with FP32 atomics.
// per chunk width PTS (64 or 128 x-points): sizes of one box row (PTS
// points x 8 channels), the stage (A: 2 M-tiles x 16 channel groups; B: 3 dx
// shifts x 2 halves) and the ring depth
template <int PTS>
struct WgCfg {
    static constexpr int BOX = PTS * 16;
    static constexpr int A_BYTES = 2 * 16 * BOX;
    static constexpr int B_BYTES = 3 * 2 * BOX;
    static constexpr int LOAD_BYTES = (9 * 2 + 3 * 2) * BOX;  // what the TMA writes per chunk
    static constexpr int STAGE = A_BYTES + B_BYTES;            // 38 / 76 KB
    static constexpr int NSTAGE = PTS == 64 ? 4 : 2;
};
constexpr int WG_THREADS = 192;
// kind::f16, D F32, A and B BF16, both MN-major (transpose bits 15, 16),
// N = 48, M = 128
constexpr unsigned IDESC_WG = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                              ((48u >> 3) << 17) | ((128u >> 4) << 24);

struct WgradArgs {
    float* dW;        // [27][ci][co], accumulated into
    float* db;        // [co] or NULL
    unsigned* status;
    int nx, ny, nz, ci, co;
};

template <int PTS>
__global__ void __launch_bounds__(WG_THREADS, 1)
    k_conv3_wgrad_tc(const __grid_constant__ CUtensorMap mx0, const __grid_constant__ CUtensorMap mx1,
                     const __grid_constant__ CUtensorMap mg0, const __grid_constant__ CUtensorMap mg1,
                     WgradArgs a)  // mx*: boxes of PTS x 3 x 1 points, mg*: PTS x 1 x 1
{
    extern __shared__ __align__(1024) unsigned char smem[];
    using C = WgCfg<PTS>;
    constexpr int WG_PTS = PTS, WG_BOX = C::BOX, WG_A_BYTES = C::A_BYTES, WG_LOAD_BYTES = C::LOAD_BYTES,
                  WG_STAGE = C::STAGE, WG_NSTAGE = C::NSTAGE;
    __shared__ __align__(8) unsigned long long full[WG_NSTAGE], empty[WG_NSTAGE], acc_full;
    __shared__ unsigned tmem_base_s;
    __shared__ volatile int abort_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ncx = a.nx / WG_PTS;
    const long long nchunks = (long long)ncx * a.ny * a.nz;

    // the ones groups (18..31: M-tile 1 after its two pair groups) of every
    // stage; the TMA never writes there
    for (int st = 0; st < WG_NSTAGE; ++st) {
        uint4* o = reinterpret_cast<uint4*>(smem + st * WG_STAGE + 18 * WG_BOX);
        const unsigned one2 = 0x3F803F80u;  // two BF16 ones
        for (int i = tid; i < 7 * 2 * WG_BOX / 16; i += WG_THREADS) o[i] = make_uint4(one2, one2, one2, one2);
    }
    if (tid == 0) {
        for (int s = 0; s < WG_NSTAGE; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&acc_full, 1);
        abort_s = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_s)),
                     "r"(128)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = tmem_base_s;
    const unsigned base = smem_u32(smem);
    int issued = 0;  // chunks whose loads thread 0 issued (for the exit drain)

    if (warp == 0) {
        if (lane == 0) {
            int i = 0;
            for (long long q = blockIdx.x; q < nchunks && !abort_s; q += gridDim.x, ++i) {
                const int s = i % WG_NSTAGE, u = i / WG_NSTAGE;
                if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1)) {
                    atomicOr(a.status, ST_TIMEOUT);
                    abort_s = 1;
                    break;
                }
                const int x0 = (int)(q % ncx) * WG_PTS;
                const int y = (int)((q / ncx) % a.ny), z = (int)(q / ((long long)ncx * a.ny));
                unsigned char* st = smem + s * WG_STAGE;
                mbar_expect_tx(&full[s], WG_LOAD_BYTES);
                for (int dz = -1; dz <= 1; ++dz) {  // rows y - 1 .. y + 1 of plane z + dz
                    tma_load_4d(st + (6 * (dz + 1)) * WG_BOX, &mx0, 0, x0, y - 1, z + dz, &full[s]);
                    tma_load_4d(st + (6 * (dz + 1) + 3) * WG_BOX, &mx1, 0, x0, y - 1, z + dz, &full[s]);
                }
                for (int g = 0; g < 3; ++g) {  // dx = g - 1: dy at q - (dx, 0, 0)
                    tma_load_4d(st + WG_A_BYTES + (2 * g) * WG_BOX, &mg0, 0, x0 - (g - 1), y, z, &full[s]);
                    tma_load_4d(st + WG_A_BYTES + (2 * g + 1) * WG_BOX, &mg1, 0, x0 - (g - 1), y, z, &full[s]);
                }
                issued = i + 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int i = 0;
            for (long long q = blockIdx.x; q < nchunks && !abort_s; q += gridDim.x, ++i) {
                const int s = i % WG_NSTAGE, u = i / WG_NSTAGE;
                if (!mbar_wait(&full[s], u & 1)) {
                    atomicOr(a.status, ST_TIMEOUT);
                    abort_s = 1;
                    break;
                }
                fence_after();
                const unsigned st = base + s * WG_STAGE;
                const unsigned long long db = smem_desc(st + WG_A_BYTES, 128, WG_BOX);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const unsigned long long da = smem_desc(st + j * 16 * WG_BOX, 128, WG_BOX);
#pragma unroll
                    for (int k = 0; k < WG_PTS / 16; ++k) {
                        // K step k = points 16k .. 16k+15 = two 8-point groups (256 B)
                        const unsigned acc = (i > 0 || k > 0) ? 1u : 0u;
                        asm volatile(
                            "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
                            "  tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem + 48 * j),
                            "l"(da + (unsigned long long)(k * 16)), "l"(db + (unsigned long long)(k * 16)),
                            "r"(IDESC_WG), "r"(acc)
                            : "memory");
                    }
                }
                mma_commit(&empty[s]);
            }
            // all issued MMAs (also after an abort) complete before acc_full
            mma_commit(&acc_full);
        }
    } else {
        // epilogue: lane quadrant q = warp % 4 -> rows 32 q + lane of each M-tile
        const int q = warp & 3;
        const bool any = (long long)blockIdx.x < nchunks;
        if (any) {
            // the lanes agree before the warp-collective TMEM loads
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_full, 0) ? 1 : 0);
            if (!ok) {
                if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
                abort_s = 1;
            } else if (__all_sync(0xffffffffu, abort_s ? 0 : 1)) {
                fence_after();
                const int r = 32 * q + lane;
                for (int j = 0; j < 2; ++j) {
                    // M row r of tile j: group gi = 16 j + r / 8 in the order
                    // (dz, half, dy) for gi < 18, then the ones (18: half 0)
                    const int gi = 16 * j + (r >> 3);
                    const int c = 8 * ((gi % 6) / 3) + (r & 7);
                    const int slot = gi < 18 ? 3 * (gi / 6) + gi % 3 : 9;  // pair (dz+1) 3 + (dy+1); 9 ones
                    const bool use = (gi < 18 && c < a.ci) || (gi == 18 && (r & 7) == 0 && a.db);
                    for (int g = 0; g < 3; ++g) {
                        // tcgen05.ld is warp-collective: every lane loads, then
                        // only the lanes with a gradient entry add it
                        float v[16];
                        tmem_ld16(tmem + ((unsigned)(32 * q) << 16) + 48 * j + 16 * g, v);
                        if (!use) continue;
                        if (slot < 9) {
                            const int t = 3 * slot + g;  // (dz+1) 9 + (dy+1) 3 + (dx+1)
                            float* w = a.dW + ((size_t)t * a.ci + c) * a.co;
                            for (int o = 0; o < a.co; ++o) atomicAdd(&w[o], v[o]);
                        } else if (g == 1) {
                            for (int o = 0; o < a.co; ++o) atomicAdd(&a.db[o], v[o]);
                        }
                    }
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    // copies still in flight after an abort land before the CTA exits
    if (abort_s && tid == 0) {
        for (int i = (issued > WG_NSTAGE ? issued - WG_NSTAGE : 0); i < issued; ++i)
            mbar_wait(&full[i % WG_NSTAGE], (i / WG_NSTAGE) & 1, 1 << 20);
    }
    if (abort_s && tid == 32) mbar_wait(&acc_full, 0, 1 << 20);
    __syncthreads();
    fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128)
                     : "memory");
}

// self-test of the bounded wait: an mbarrier nobody arrives at; the wait
// must give up after `polls` polls and record ST_TIMEOUT
__global__ void k_selftest_wait(unsigned* status, long long polls)
{
    // two barriers nobody arrives on: the convolutions' wait and the
    // stencil's bulk-copy wait (ls_stencil.cuh) must both give up
    __shared__ __align__(8) unsigned long long bar[2];
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool a = mbar_wait(&bar[0], 0, polls);
        const bool b = bulk_wait(smem_u32(&bar[1]), 0, polls);
        if (!a && !b) atomicOr(status, ST_TIMEOUT);
    }
}

// pack W (FP32 [27][ci][co], ci, co <= 16) into the canonical K-major B
// layout per (dx, dy) shift p = (dy + 1) 3 + (dx + 1): [kb][nb][8 n][8 k]
// bf16 with N = 48 rows n = 16 g + o (g = dz + 1) and K = 16:
// B[n][k] = W[t][k][o], t = 9 g + p.  flip: the backward-data operator,
// B[n][k] = W[26 - t][o][k] (taps mirrored, channels swapped).  Missing
// channels are zero.
__global__ void k_pack_weights(const float* __restrict__ W, int ci, int co, int flip,
                               __nv_bfloat16* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // over 9 * 768 entries
    if (i >= 9 * 768) return;
    const int p = i / 768, r = i % 768;
    const int kb = r / 384, nb = (r / 64) % 6, n8 = (r / 8) % 8, k8 = r % 8;
    const int n = nb * 8 + n8, k = kb * 8 + k8;
    const int g = n / 16, o = n % 16, t = 9 * g + p;
    float v = 0.f;
    if (!flip) {
        if (k < ci && o < co) v = W[((size_t)t * ci + k) * co + o];
    } else {
        // forward weights W[t][c][o'] with c < ci, o' < co; here k = o', o = c
        if (o < ci && k < co) v = W[((size_t)(26 - t) * ci + o) * co + k];
    }
    out[i] = __float2bfloat16_rn(v);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

}  // namespace

bool conv3_shape_ok(int nx, int ny, int nz)
{
    return nx >= BXP && nx % BXP == 0 && ny >= BYP && ny % BYP == 0 && nz >= BZP && nz % BZP == 0;
}

// tensor maps over act[nz][ny][nx][16] bf16 viewed as (8 channels, x, y, z):
// map[h] covers channels 8h..8h+7 (base address + 16 h bytes); box of
// bx x by x bz points
static cudaError_t make_maps_box(CUtensorMap* maps, const void* act, int nx, int ny, int nz, int bx,
                                 int by, int bz)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    if (((uintptr_t)act & 15u) != 0) return cudaErrorInvalidValue;
    const cuuint64_t dims[4] = {8, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[3] = {32, (cuuint64_t)32 * nx, (cuuint64_t)32 * nx * ny};
    const cuuint32_t box[4] = {8, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int h = 0; h < 2; ++h) {
        CUresult r = fn(&maps[h], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4,
                        (void*)((const char*)act + 16 * h), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

cudaError_t make_act_maps(CUtensorMap* maps, const void* act, int nx, int ny, int nz)
{
    return make_maps_box(maps, act, nx, ny, nz, PX, PY, PZ);
}

int conv3_blocks(int nx, int ny, int nz) { return (nx / BXP) * (ny / BYP) * (nz / BZP); }

bool conv3_wgrad_shape_ok(int nx, int ny, int nz)
{
    return nx >= 64 && nx % 64 == 0 && ny >= 1 && nz >= 1;
}

template <int PTS>
static cudaError_t launch_wgrad_pts(const void* x, const void* dy, int nx, int ny, int nz, int ci,
                                    int co, float* dW, float* db, unsigned* status, cudaStream_t s)
{
    using C = WgCfg<PTS>;
    CUtensorMap mx[2], mg[2];
    cudaError_t e = make_maps_box(mx, x, nx, ny, nz, PTS, 3, 1);
    if (e != cudaSuccess) return e;
    e = make_maps_box(mg, dy, nx, ny, nz, PTS, 1, 1);
    if (e != cudaSuccess) return e;
    static bool attr = false;
    const int smem = C::NSTAGE * C::STAGE;
    if (!attr) {
        e = cudaFuncSetAttribute(k_conv3_wgrad_tc<PTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    WgradArgs a;
    a.dW = dW;
    a.db = db;
    a.status = status;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.ci = ci;
    a.co = co;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long nchunks = (long long)(nx / PTS) * ny * nz;
    const int grid = (int)(nchunks < sms ? nchunks : sms);
    k_conv3_wgrad_tc<PTS><<<grid, WG_THREADS, smem, s>>>(mx[0], mx[1], mg[0], mg[1], a);
    return cudaGetLastError();
}

cudaError_t launch_conv3_wgrad(const void* x, const void* dy, int nx, int ny, int nz, int ci,
                               int co, float* dW, float* db, unsigned* status, cudaStream_t s)
{
    if (!conv3_wgrad_shape_ok(nx, ny, nz) || ci < 1 || ci > 16 || co < 1 || co > 16)
        return cudaErrorInvalidValue;
    // chunks of 128 points where the rows allow: half the TMA boxes per point
    if (nx % 128 == 0) return launch_wgrad_pts<128>(x, dy, nx, ny, nz, ci, co, dW, db, status, s);
    return launch_wgrad_pts<64>(x, dy, nx, ny, nz, ci, co, dW, db, status, s);
}

cudaError_t launch_selftest_wait(unsigned* status, long long polls, cudaStream_t s)
{
    k_selftest_wait<<<1, 32, 0, s>>>(status, polls);
    return cudaGetLastError();
}

cudaError_t launch_pack_weights(const float* W, int ci, int co, int flip, void* out, cudaStream_t s)
{
    k_pack_weights<<<(9 * 768 + 255) / 256, 256, 0, s>>>(W, ci, co, flip, (__nv_bfloat16*)out);
    return cudaGetLastError();
}

cudaError_t launch_conv3(const CUtensorMap* maps, const void* wpack, const float* bias,
                         const void* mask, void* out_bf16, float* out_f32, int nx, int ny, int nz,
                         int mode, unsigned* status, cudaStream_t s, const int* blist,
                         const int* bcount)
{
    static bool attr = false;
    const int smem = NSTAGE * XS_BYTES + W_BYTES;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_conv3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    ConvArgs a;
    a.wpack = (const __nv_bfloat16*)wpack;
    a.bias = bias;
    a.mask = (const __nv_bfloat16*)mask;
    a.out_bf16 = (__nv_bfloat16*)out_bf16;
    a.out_f32 = out_f32;
    a.status = status;
    a.blist = blist;
    a.bcount = blist ? bcount : nullptr;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.mode = mode;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // with a list the grid covers every block (the count is on the device)
    const int nblocks = conv3_blocks(nx, ny, nz);
    int grid = sms;
    if (grid > nblocks) grid = nblocks;
    k_conv3_tc<<<grid, CONV_THREADS, smem, s>>>(maps[0], maps[1], a);
    return cudaGetLastError();
}

}  // namespace lsk
