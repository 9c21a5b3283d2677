// ls_internal.cuh -- device-side data model shared by the library's kernels
// and its host engine.
//
// Storage ("bricked") layout in HBM: every 8x8x8 tile is one contiguous
// block of 512 values (2 KiB in FP32, 4 KiB in FP64); inside a tile the order
// is (lz*8 + ly)*8 + lx, x fastest.  Tile t of instance i starts at element
// (tile_base_i + t) * 512.  A tile is thus one DRAM-contiguous burst and the
// stencil's face halos are 256-byte (z) or 32-byte (y) runs of the
// neighbouring tiles.  Row-major arrays crossing the ABI are converted on
// the device by the pack / unpack kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lsk {

constexpr int TILE = 8;
constexpr int TILE_PTS = TILE * TILE * TILE;
constexpr int XFACE_FLOATS = 2 * TILE * TILE;  // two x-faces of one tile

// Per-instance parameters (one entry per independent grid).
struct Inst {
    int nx, ny, nz;        // grid points (multiples of 8)
    int tnx, tny, tnz;     // tiles per axis
    long long tile_base;   // global id of the instance's tile 0
    long long ntiles;      // tnx * tny * tnz
    double h;              // grid spacing
    double inv_h;          // 1/h
    double gamma;          // band threshold halfwidth * h (FP64)
    double Fc;             // constant speed when speed_mode == 1
    int speed_mode;        // 0: unset, 1: constant, 2: field
    int pow2h;             // h is a power of two (1/h exact)
    int bc;                // 0 extrapolate, 1 neumann
    int ghost;             // slab split: bit 0 / bit 1 = the bottom / top tile row
                           // holds a neighbour's copy (never active)
};

// Device status word bits (sticky).
enum : unsigned {
    ST_TIMEOUT = 1u,
    ST_BOUNDS = 2u,
    ST_NONFINITE = 4u,
};

// Per-active-tile info byte written by the rebuild (read by the stencil, so
// that it needs no tile-coordinate arithmetic): which of the six face
// neighbours exist inside the instance, and whether every speed of the tile
// has one sign.
enum : unsigned {
    NB_XM = 1u, NB_XP = 2u, NB_YM = 4u, NB_YP = 8u, NB_ZM = 16u, NB_ZP = 32u,
    NB_ALL = 63u,
    SG_POS = 64u,   // every F >= 0 in the tile (G+ of Eq. 4 everywhere)
    SG_NEG = 128u,  // every F < 0 in the tile (G- of Eq. 5 everywhere)
    // list_nact bits above the NB_* bits: the x-face copy of the frozen
    // -x / +x neighbour is still to be written (StepArgs::xface_fill)
    NACT_FILL_XM = NB_XM << 6, NACT_FILL_XP = NB_XP << 6,
};

// Per-step scalars on the device, one per instance.
struct StepScalars {
    double M;      // max |F| over the active set at the last rebuild
    double dt;     // current time step
    float coef;    // (float)(dt / h), FP32 path
    int active;    // active tiles of this instance at the last rebuild (batched)
    float Fc;      // (float) constant speed, FP32 path (batched: read per tile)
};

// ---------------------------------------------------------------------------
// launchers (ls_band.cu)
// ---------------------------------------------------------------------------
// row-major <-> bricked conversion of one instance; counts non-finite values
// into *nonfinite (may be NULL)
cudaError_t launch_pack(const void* src, void* dst, const Inst& in, int prec, unsigned* nonfinite,
                        cudaStream_t s);
// device-to-device copy of `bytes` (a multiple of 16, 16-byte aligned; also
// into dst2 when it is not NULL: one read, two writes) by a
// kernel, so that it does not queue behind host transfers on a copy engine
cudaError_t launch_copy(void* dst, const void* src, size_t bytes, cudaStream_t s,
                        void* dst2 = nullptr);
cudaError_t launch_unpack(const void* src, void* dst, const Inst& in, int prec, cudaStream_t s);
// tile_maxF[t] = max |F| over tile t; tile_sgn[t] = SG_POS / SG_NEG / 0
cudaError_t launch_tile_speed(const void* F, void* tile_maxF, uint8_t* tile_sgn, long long ntiles,
                              int prec, cudaStream_t s);
// core[t] = (min_{p in t} |phi_p| < gamma) over all tiles of all instances
cudaError_t launch_classify_all(const void* phi, uint8_t* core, const Inst* d_inst,
                                const uint16_t* tile_inst, const Inst& single, long long ntiles,
                                int prec, cudaStream_t s);
// band rebuild: dilation by one tile over 26 or 6 neighbours (conn; act bit
// 0 = new flag, bit 1 = previous) + block counts, turned into exclusive
// offsets and the active count *count by the last block to finish (done: a
// zeroed device counter, reset by that block)
// dst + t * dst_stride <- src + t * src_stride, `words` 32-bit words per
// chunk, t < nchunks (strides in words)
cudaError_t launch_chunk_copy(const void* src, long long src_stride_words, void* dst,
                              long long dst_stride_words, int words, long long nchunks, cudaStream_t s);
// sc[0].M = *Mext, then dt = cfl h / M as at a rebuild (single grid)
cudaError_t launch_set_dt_from(StepScalars* sc, const double* Mext, const Inst& in, double cfl,
                               int prec, cudaStream_t s);
// per tile row (tz) count of the active-list entries: rows[tz] += 1
cudaError_t launch_row_counts(const int* list, const int* count, int tiles_per_row, int* rows,
                              int capacity, cudaStream_t s);
cudaError_t launch_dilate(const uint8_t* core, uint8_t* act, int* block_counts,
                          const Inst* d_inst, const uint16_t* tile_inst, const Inst& single,
                          long long ntiles, unsigned* done, int* count, int conn,
                          cudaStream_t s);
// exclusive scan of block counts, writes total to *count
cudaError_t launch_scan(int* block_counts, int nblocks, int* count, cudaStream_t s);
// local scheme: the active-list entries whose tile holds a point of N
// (nflag), compacted in ascending order with their info bytes and N bits
// (block counts, scanned by the last block -> scatter); core[t] = 0 for the
// others when core is not NULL
cudaError_t launch_nflag_count(const uint8_t* nflag, const int* count, int* block_counts,
                               int nblocks, unsigned* done, int* total, cudaStream_t s);
cudaError_t launch_nflag_scatter(const uint8_t* nflag, const int* count, const int* block_offsets,
                                 const int* list, const uint8_t* list_info, const uint32_t* nmask,
                                 int* nl, uint8_t* nl_info, uint32_t* nl_mask, uint8_t* core,
                                 int nblocks, cudaStream_t s);
// scatter active ids (ascending) with their info bytes, fold max |F| of the
// active tiles into *Mbits (ordered bits of a non-negative float / double),
// and copy the tiles leaving the active set from cur into other; the last
// block to finish sets the step scalars (dt from M as launch_set_dt with
// finalize = 1; done: a zeroed device counter).
// tile_sgn == NULL: constant speed, sign bits const_sgn.
// list_nact (may be NULL): per entry, the face neighbours inside the domain
// that are active (NB_* bits)
cudaError_t launch_scatter(const uint8_t* act, const int* block_offsets, int* list,
                           uint8_t* list_info, const uint8_t* tile_sgn, unsigned const_sgn,
                           const Inst& single, long long ntiles, const void* tile_maxF, int prec,
                           unsigned long long* Mbits, const void* cur, void* other,
                           uint8_t* list_nact, StepScalars* sc, int dt_mode, double dt_value,
                           const int* count, unsigned* done, int xface_mode, cudaStream_t s);
// full-domain list: every tile, ascending, with info bytes; *count = ntiles
cudaError_t launch_full_list(int* list, uint8_t* list_info, const uint8_t* tile_sgn,
                             unsigned const_sgn, const Inst& single, long long ntiles, int* count,
                             uint8_t* list_nact, cudaStream_t s);
// max of tile max|F| over all tiles (full-domain mode)
cudaError_t launch_max_all(const void* tile_maxF, long long ntiles, int prec,
                           unsigned long long* Mbits, cudaStream_t s);
// dt from M (FP64): mode 0 fixed (value = dt), 1 CFL (value = CFL number).
// finalize = 1: M is taken from *Mbits (or |Fc| for a constant speed) and
// *Mbits cleared; count (device) or fixed_count = number of active tiles.
cudaError_t launch_set_dt(StepScalars* sc, int n_inst, const Inst* d_inst, const Inst& single,
                          int mode, double value, int finalize, int prec,
                          unsigned long long* Mbits, const int* count, long long fixed_count,
                          cudaStream_t s);

// ---------------------------------------------------------------------------
// launchers (ls_step.cu)
// ---------------------------------------------------------------------------
// Passes of the local scheme (section 1.1, Steps 1-3).  One step is OP_CUT
// (Eq. 8 as Eq. 3 with the speed c(|phi|) F, writing the mask of N of
// Eq. 11) and then K passes OP_REINIT (one pseudo-time iteration of Eq. 12
// on N), the last one OP_REINIT_CLAMP (plus Eq. 10 on N); with K = 0 the
// advance is OP_CUT_CLAMP.
enum : int { OP_PLAIN = 0, OP_CUT = 1, OP_CUT_CLAMP = 2, OP_REINIT = 3, OP_REINIT_CLAMP = 4 };

struct LocalParams {
    double beta, gamma;   // Eq. 7 thresholds (FP64)
    double dtau;          // pseudo-time step of Eq. 12
    float beta_dn;        // largest float <= beta (the FP32 kernels no longer test it;
                          // without it the parameter block measured slower for the
                          // reinitialisation pass, 35.3 against 34.9 us)
    float gamma_up;       // smallest float >= gamma: FP32 |phi| < gamma decided as in FP64,
                          // and the clamp bound (a clamped value is not in T)
    float beta_n, gamma_n;  // nearest floats (the cubic of Eq. 7)
    float inv_w;          // 1 / (gamma - beta)
    float lam;            // dtau / h
    float dtau_f;         // dtau
    int pad;
};

struct StepArgs {
    const void* src;
    void* dst;
    const void* F;            // field (bricked) or NULL for constant speed
    const int* list;          // active tile ids (ascending)
    const uint8_t* info;      // per-entry info byte (NB_* | SG_*)
    const uint16_t* list_inst;  // per-entry instance (batched contexts), else NULL
    const int* count;         // number of active tiles (device)
    const StepScalars* sc;    // per-instance dt, dt/h
    const Inst* insts;        // per-instance parameters (batched), device
    uint8_t* core;            // fused tube test output, or NULL
    unsigned long long* updates;
    unsigned long long* updates_timed;  // also counts this launch's updates when the
                                        // profile times it (else NULL)
    unsigned long long* updates2;  // two-step passes: points passed (each updated twice)
    Inst in;                  // single instance parameters (bc is read from here always)
    int max_grid;             // cap on the persistent grid (0 = none)
    int reverse;              // FP32: walk the list from its end (L2 reuse across launches)
    int early;                // the previous launch was a step over the same list and
                              // dt: the list, its count and the scalars may be read
                              // before the wait for that launch (one-warp kernel)
    const uint8_t* tile_sgn;  // full-domain column kernel: per-tile sign class of F, or NULL
    // local scheme (single instance, 4 points per thread)
    int op;                   // OP_*
    LocalParams lp;
    uint32_t* nmask;          // N of Eq. 11: 16 words (512 bits) per list entry
    uint8_t* nflag;           // advance: per entry, 1 when the tile holds a point of N
    const uint8_t* nact;      // per entry: face neighbours inside the domain that are
                              // active (NB_* bits; breach test)
    unsigned long long* breaches;  // N points found in inactive tiles
    // FP32 plain step, single grid: copies of the x-faces of the entries'
    // frozen x neighbours (inside the domain, not active: bits of nact),
    // XFACE_FLOATS per tile id, [side][lz][ly] (side 0: the x = 7 column of
    // tile t - 1, side 1: the x = 0 column of tile t + 1).  A frozen tile
    // keeps its values until the next rebuild, so the copy is read in 256-byte
    // runs by every step instead of one 32-byte sector per value.  NULL: every
    // x-halo value is read from the neighbour tile.
    float* xface;
    // 1: faces whose NACT_FILL bit is set are read from the neighbour and
    // their copy written (the first plain step after a rebuild)
    int xface_fill;
    unsigned* status;         // sticky device status word (ST_*)
};

// launch configuration of the FP32 stencil, chosen by the autotuner
struct StepConfig {
    int stages = 3;           // cp.async ring depth (2, 3, 4)
    int grid_pct = 100;       // persistent grid, percent of full occupancy
    int ppt = 4;              // points per thread: 4 (128-thread CTAs), 8 (64-thread CTAs) or
                              // 16 (one warp per tile, ls_step_z4.cu)
    int spp = 1;              // steps per pass: 1, or 2 (temporal blocking, ls_step2.cu)
    int grid_pct2 = 100;      // persistent grid of the two-step passes
    int dense = 0;            // full domain: the column-streaming kernel (ls_dense.cu)
};

cudaError_t launch_step(const StepArgs& a, int prec, const StepConfig& cfg, cudaStream_t s);
// FP32 plain step with one warp per tile, 16 points per thread (ls_step_z4.cu)
cudaError_t launch_step_z4(const StepArgs& a, const StepConfig& cfg, cudaStream_t s);
// FP32 cut-off advance of the local scheme (a.op = OP_CUT / OP_CUT_CLAMP)
// with one warp per tile (ls_local_z4.cu)
cudaError_t launch_local_z4(const StepArgs& a, const StepConfig& cfg, cudaStream_t s);
// FP64 step and local-scheme passes (ls_step64.cu)
cudaError_t launch_step64(const StepArgs& a, cudaStream_t s);
// two steps per pass (FP32 single grid, plain scheme; a.nact required);
// grid from cfg.grid_pct2
cudaError_t launch_step2(const StepArgs& a, const StepConfig& cfg, cudaStream_t s);
// full-domain mode, FP32 single grid, plain scheme: tile columns streamed
// along z (ls_dense.cu); every tile, no list
cudaError_t launch_dense_step(const StepArgs& a, const StepConfig& cfg, cudaStream_t s);

// ---------------------------------------------------------------------------
// batched rebuild helpers (ls_band.cu)
// ---------------------------------------------------------------------------
// scatter for a batch: list + info + instance id per entry; per-instance
// active counts and max|F| bits; leaving-tile copy
cudaError_t launch_scatter_batch(const uint8_t* act, const int* block_offsets, int* list,
                                 uint8_t* list_info, uint16_t* list_inst,
                                 const uint8_t* tile_sgn, const Inst* d_inst,
                                 const uint16_t* tile_inst, long long ntiles,
                                 const void* tile_maxF, int prec, unsigned long long* Mbits,
                                 int* inst_count, const void* cur, void* other, cudaStream_t s);
// per-instance dt from per-instance M (finalize: from Mbits / |Fc| and the
// per-instance active counts, then clear both)
// incremental rebuild (the steps since the previous rebuild ran
// the fused tube test): marks from the core entries of the previous list,
// their count and scan, the ascending ids + act + the leaving tiles' ids,
// and the entries' info bytes, instances, per-instance counts and max |F|
// with the leaving tiles' copies (leave: ntiles ints, nleave: one int).  The
// flag arrays act and mark hold whole 16-byte chunks (zero padding); mark
// is zero between rebuilds.
cudaError_t launch_mark(const int* list, const int* count, const uint8_t* core, uint8_t* mark,
                        const Inst* d_inst, const uint16_t* tile_inst, const Inst& single,
                        long long ntiles, int conn, cudaStream_t s);
cudaError_t launch_mark_count(const uint8_t* mark, long long ntiles, int* block_counts,
                              unsigned* done, int* count, int* nleave, cudaStream_t s);
cudaError_t launch_mark_scatter(uint8_t* mark, uint8_t* act, long long ntiles,
                                const int* block_offsets, int* list, int* leave, int* nleave,
                                cudaStream_t s);
cudaError_t launch_entry_batch(const int* list, const int* count, uint8_t* list_info,
                               uint16_t* list_inst, const uint8_t* tile_sgn, const Inst* d_inst,
                               const uint16_t* tile_inst, long long ntiles, const void* tile_maxF,
                               int prec, unsigned long long* Mbits, int* inst_count,
                               const int* leave, const int* nleave, const void* cur, void* other,
                               cudaStream_t s);
// single grid: info bytes, active / frozen-face bytes (xface_mode as
// launch_scatter), max |F|, the leaving tiles' copies, dt in the last block
cudaError_t launch_entry_single(const int* list, const int* count, uint8_t* list_info,
                                const uint8_t* act, const uint8_t* tile_sgn, unsigned const_sgn,
                                const Inst& single, long long ntiles, const void* tile_maxF, int prec,
                                unsigned long long* Mbits, uint8_t* list_nact, int xface_mode,
                                const int* leave, const int* nleave, const void* cur, void* other,
                                StepScalars* sc, int dt_mode, double dt_value, unsigned* done,
                                cudaStream_t s);
cudaError_t launch_set_dt_batch(StepScalars* sc, int n_inst, const Inst* d_inst, int mode,
                                double value, int finalize, int prec, unsigned long long* Mbits,
                                int* inst_count, cudaStream_t s);

// ---------------------------------------------------------------------------
// learned corrector (ls_conv.cu, ls_learned.cu)
// ---------------------------------------------------------------------------
// blocks of 8 x 16 x 4 points: nx a multiple of 8, ny of 16, nz of 4
bool conv3_shape_ok(int nx, int ny, int nz);
int conv3_blocks(int nx, int ny, int nz);
cudaError_t make_act_maps(CUtensorMap* maps, const void* act, int nx, int ny, int nz);
// the convolution blocks (ids bx + nbx (by + nby bz)) whose tiles lie within
// one tile of an active tile (act bit 0) of a single grid; unordered
cudaError_t launch_block_list(const uint8_t* act, const Inst& in, int* list, int* count,
                              cudaStream_t s);
cudaError_t launch_pack_weights(const float* W, int ci, int co, int flip, void* out, cudaStream_t s);
// mode 0: out_bf16 = relu(conv + b); 1: out_f32 = (conv + b) channel 0;
// 2: out_bf16 = conv(x) * [mask > 0] (x: gradient, weights packed flipped)
cudaError_t launch_conv3(const CUtensorMap* maps, const void* wpack, const float* bias,
                         const void* mask, void* out_bf16, float* out_f32, int nx, int ny, int nz,
                         int mode, unsigned* status, cudaStream_t s, const int* blist = nullptr,
                         const int* bcount = nullptr);
cudaError_t launch_features(const float* phi, const float* phit, const float* F, float Fc,
                            float inv_h, long long n, void* X, cudaStream_t s);
cudaError_t launch_features_bricked(const float* phi, const float* phit, const float* F,
                                   const Inst& in, void* X, cudaStream_t s);
cudaError_t launch_count_mask(const float* phi, double gamma, long long n, int* count, cudaStream_t s);
cudaError_t launch_loss_grad(const float* z, const float* phi, const float* phit,
                             const float* phiref, float inv_h, double gamma, const int* count,
                             long long n, void* dz, double* loss, cudaStream_t s);
// dW [27][ci][co] += sum_p x[p + off(tap)] dy[p], db += sum_p dy[p] (db may
// be NULL) on the tensor cores; nx a multiple of 64
bool conv3_wgrad_shape_ok(int nx, int ny, int nz);
cudaError_t launch_conv3_wgrad(const void* x, const void* dy, int nx, int ny, int nz, int ci,
                               int co, float* dW, float* db, unsigned* status, cudaStream_t s);
cudaError_t launch_adam(float* w, const float* g, float* m, float* v, int n, float lr, int step,
                        cudaStream_t s);
cudaError_t launch_residual(float* phit, const float* z, const int* list, const int* count,
                            const Inst& in, const StepScalars* sc, float hc, unsigned* flag,
                            unsigned long long* fallbacks, cudaStream_t s);
cudaError_t launch_restrict4(const float* fine, int nfx, int nfy, int nfz, float* coarse,
                             cudaStream_t s);
cudaError_t launch_selftest_wait(unsigned* status, long long polls, cudaStream_t s);
// Step 0 fields (ls_init.cu): evaluate shape / speed `kind` with device
// params into out (and out2 if not NULL), bricked, context precision
cudaError_t launch_init_field(void* out, void* out2, const Inst& in, int prec, int is_speed,
                              int kind, const double* params, cudaStream_t s);

}  // namespace lsk
