// ls_api.cu -- the C ABI (include/ls.h) and the host engine behind it: the
// context, its device buffers, and the rebuild / step schedule of the
// narrow-band algorithm (section 1.1, Steps 1-2).
//
// Schedule, per step of ls_step:
//   1. band stale (after ls_set_phi / ls_set_speed*) -> full rebuild: tube
//      test on every tile;  rebuild_every steps since the last rebuild ->
//      rebuild from the tube flags that the previous step computed on the
//      tiles it updated (inactive tiles are frozen and were outside the tube
//      at the last rebuild, so they cannot have entered it);
//   2. rebuild = dilation -> scan of block counts -> ascending scatter of
//      active ids with their info bytes, folding max|F| of the active tiles
//      and copying tiles that leave the active set into the other ping-pong
//      buffer -> dt in FP64;
//   3. one launch of the stencil over the active list, src -> dst, swap.
// Nothing is read back to the host inside ls_step: counts, M and dt stay in
// device memory and the persistent stencil grid reads the count there, so a
// whole ls_step call can be captured once as a CUDA graph and replayed.
//
// A batched context holds n independent grids in one set of buffers: the
// tiles of instance i occupy global tile ids [tile_base_i, tile_base_i +
// ntiles_i); one rebuild and one stencil launch per step serve every
// instance through a single global active-tile queue, with per-instance dt,
// speed and band threshold.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ls_ctx.cuh"

using lsk::GraphEntry;
using lsk::GraphKey;
using lsk::SchedState;

static thread_local int g_last_cuda_error = 0;

namespace {

int cuda_fail(cudaError_t e)
{
    g_last_cuda_error = (int)e;
    if (e == cudaErrorMemoryAllocation) return LS_ENOMEM;
    return LS_ECUDA;
}

#define CK(expr)                                     \
    do {                                             \
        cudaError_t e_ = (expr);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

// a library kernel launch: counted, then checked
#define KL(c, expr)      \
    do {                 \
        ++(c)->launches; \
        CK(expr);        \
    } while (0)

#define RET(expr)                \
    do {                         \
        int r_ = (expr);         \
        if (r_ != LS_OK) return r_; \
    } while (0)

cudaError_t take_event(ls_ctx* c, cudaEvent_t* e)
{
    if (!c->ev_free.empty()) {
        *e = c->ev_free.back();
        c->ev_free.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(e);
}

// fold finished event pairs into stencil_ms (synchronises the stream)
int drain_events(ls_ctx* c)
{
    if (c->ev_pending.empty()) return LS_OK;
    CK(cudaStreamSynchronize(c->stream));
    for (auto& p : c->ev_pending) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, p.e0, p.e1));
        c->stencil_ms += ms;
        c->stencil_timed += (unsigned long long)p.count;
        if (p.reinit) {
            c->reinit_ms += ms;
            c->reinit_timed += (unsigned long long)p.count;
        }
        c->ev_free.push_back(p.e0);
        c->ev_free.push_back(p.e1);
    }
    c->ev_pending.clear();
    return LS_OK;
}

void clear_graphs(ls_ctx* c)
{
    for (auto& kv : c->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    c->graphs.clear();
}

// any change of state that kernels read by value (or that changes the launch
// sequence) invalidates the cached graphs
void state_changed(ls_ctx* c)
{
    c->band_valid = false;
    c->core_fresh = false;
    clear_graphs(c);
}

bool is_pow2(double h)
{
    int e = 0;
    return std::frexp(h, &e) == 0.5;
}

template <typename T>
cudaError_t dalloc(T** p, size_t bytes)
{
    return cudaMalloc((void**)p, bytes ? bytes : 16);
}

void free_all(ls_ctx* c)
{
    clear_graphs(c);
    for (auto& p : c->ev_pending) {
        cudaEventDestroy(p.e0);
        cudaEventDestroy(p.e1);
    }
    for (auto e : c->ev_free) cudaEventDestroy(e);
    void* ptrs[] = {c->phi[0], c->phi[1], c->F, c->tile_maxF, c->tile_sgn, c->staging, c->snapshot, c->core,
                    c->act, c->mark, c->d_leave, c->d_nleave, c->list, c->list_info, c->d_count, c->block_counts, c->d_sc,
                    c->d_Mbits, c->d_updates, c->d_status, c->d_inst,
                    c->d_tile_inst, c->d_list_inst, c->d_inst_count, c->init_params, c->nmask,
                    c->d_breaches, c->list_nact, c->nmask2, c->nflag, c->nl, c->nl_info,
                    c->d_ncount, c->d_rupdates, c->d_done, c->d_updates2, c->xface,
                    c->d_updates_timed, c->d_rowcnt};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->h_nonfinite) cudaFreeHost(c->h_nonfinite);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    if (c->learned) lsk::learned_free(c->learned);
    c->learned = nullptr;
    if (c->output) lsk::output_free(c->output);
    c->output = nullptr;
    if (c->hio) {
        lsk::HostIO* H = c->hio;
        if (H->h2d) cudaStreamSynchronize(H->h2d);
        if (H->d2h) cudaStreamSynchronize(H->d2h);
        for (cudaEvent_t e : {H->staged, H->consumed, H->unpacked, H->drained})
            if (e) cudaEventDestroy(e);
        for (void* p : {H->in_phi, H->in_F, H->out})
            if (p) cudaFree(p);
        if (H->h2d) cudaStreamDestroy(H->h2d);
        if (H->d2h) cudaStreamDestroy(H->d2h);
        delete H;
        c->hio = nullptr;
    }
}

size_t grid_bytes(const ls_ctx* c) { return c->npts * c->esize; }
size_t inst_bytes(const ls_ctx* c, const Inst& in) { return (size_t)in.ntiles * lsk::TILE_PTS * c->esize; }
char* region(const ls_ctx* c, void* buf, const Inst& in)
{
    return (char*)buf + (size_t)in.tile_base * lsk::TILE_PTS * c->esize;
}

int ensure_staging(ls_ctx* c)
{
    if (!c->staging) CK(dalloc(&c->staging, c->max_inst_pts * c->esize));
    return LS_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int upload_insts(ls_ctx* c)
{
    if (c->batched)
        CK(cudaMemcpyAsync(c->d_inst, c->insts.data(), sizeof(Inst) * c->n_inst,
                           cudaMemcpyHostToDevice, c->stream));
    return LS_OK;
}

// pack a row-major source (host or device) of instance `in` into the bricked
// buffer dst (already offset to the instance); LS_ENONFINITE if any value is
// NaN/Inf (after a stream sync)
int pack_from(ls_ctx* c, const Inst& in, const void* src, int on_device, void* dst)
{
    const void* dsrc = src;
    if (!on_device) {
        RET(ensure_staging(c));
        CK(cudaMemcpyAsync(c->staging, src, inst_bytes(c, in), cudaMemcpyHostToDevice, c->stream));
        dsrc = c->staging;
    } else if (!aligned16(src)) {
        return LS_EINVAL;
    }
    // the flag is a mapped host word: no copy-engine transfer, so the check
    // does not wait behind a read-back in flight on another stream
    volatile unsigned* flag = c->h_nonfinite;
    *flag = 0u;
    KL(c, lsk::launch_pack(dsrc, dst, in, c->prec, c->d_nonfinite, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return *flag ? LS_ENONFINITE : LS_OK;
}

unsigned const_sign_bits(const ls_ctx* c) { return c->insts[0].Fc >= 0.0 ? lsk::SG_POS : lsk::SG_NEG; }

int speed_mode(const ls_ctx* c)
{
    // one mode for every instance (0 if unset or mixed)
    const int m = c->insts[0].speed_mode;
    for (const Inst& in : c->insts)
        if (in.speed_mode != m) return 0;
    return m;
}

const uint8_t* sign_table(const ls_ctx* c) { return speed_mode(c) == 2 ? c->tile_sgn : nullptr; }

// incr: the band was valid before this rebuild (no value changed since the
// previous one other than by the steps)
int finish_rebuild(ls_ctx* c, bool incr, cudaStream_t s)
{
    // the frozen x-face copies: only the new faces are filled when every face
    // of the previous band was (a filling step ran since that rebuild)
    const int xmode = c->xface ? (incr && !c->xface_pending ? 2 : 1) : 0;
    void* cur = c->phi[c->cur];
    void* other = c->phi[c->cur ^ 1];
    const void* tmf = speed_mode(c) == 2 ? c->tile_maxF : nullptr;
    if (c->batched) {
        KL(c, lsk::launch_scatter_batch(c->act, c->block_counts, c->list, c->list_info,
                                        c->d_list_inst, sign_table(c), c->d_inst, c->d_tile_inst,
                                        c->ntiles, tmf, c->prec, c->d_Mbits, c->d_inst_count, cur,
                                        other, s));
        KL(c, lsk::launch_set_dt_batch(c->d_sc, c->n_inst, c->d_inst, c->dt_mode, c->dt_value, 1,
                                       c->prec, c->d_Mbits, c->d_inst_count, s));
    } else {
        KL(c, lsk::launch_scatter(c->act, c->block_counts, c->list, c->list_info, sign_table(c),
                                  const_sign_bits(c), c->in0(), c->ntiles, tmf, c->prec,
                                  c->d_Mbits, cur, other, c->list_nact, c->d_sc, c->dt_mode,
                                  c->dt_value, c->d_count, c->d_done + 1, xmode, s));
        c->xface_pending = xmode != 0;
    }
    return LS_OK;
}

// an NVTX range around a host-side phase (visible to nsys / ncu timelines;
// a no-op without a tool attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// the incremental rebuild: the new active set marked from the core entries
// of the previous list (core is fresh on every entry and 0 on the other
// tiles), then compacted 16 tiles per thread; the list, the flags, the
// frozen x-face bits, M and dt are those of the full scan
int rebuild_incr(ls_ctx* c, bool incr, cudaStream_t s)
{
    void* cur = c->phi[c->cur];
    void* other = c->phi[c->cur ^ 1];
    const void* tmf = speed_mode(c) == 2 ? c->tile_maxF : nullptr;
    KL(c, lsk::launch_mark(c->list, c->d_count, c->core, c->mark, c->dinst(), c->tinst(), c->in0(),
                           c->ntiles, c->dilation, s));
    KL(c, lsk::launch_mark_count(c->mark, c->ntiles, c->block_counts, c->d_done, c->d_count,
                                 c->d_nleave, s));
    KL(c, lsk::launch_mark_scatter(c->mark, c->act, c->ntiles, c->block_counts, c->list, c->d_leave,
                                   c->d_nleave, s));
    if (c->batched) {
        KL(c, lsk::launch_entry_batch(c->list, c->d_count, c->list_info, c->d_list_inst, sign_table(c),
                                      c->d_inst, c->d_tile_inst, c->ntiles, tmf, c->prec, c->d_Mbits,
                                      c->d_inst_count, c->d_leave, c->d_nleave, cur, other, s));
        KL(c, lsk::launch_set_dt_batch(c->d_sc, c->n_inst, c->d_inst, c->dt_mode, c->dt_value, 1,
                                       c->prec, c->d_Mbits, c->d_inst_count, s));
    } else {
        const int xmode = c->xface ? (incr && !c->xface_pending ? 2 : 1) : 0;
        KL(c, lsk::launch_entry_single(c->list, c->d_count, c->list_info, c->act, sign_table(c),
                                       const_sign_bits(c), c->in0(), c->ntiles, tmf, c->prec,
                                       c->d_Mbits, c->list_nact, xmode, c->d_leave, c->d_nleave, cur,
                                       other, c->d_sc, c->dt_mode, c->dt_value, c->d_done + 1, s));
        c->xface_pending = xmode != 0;
    }
    return LS_OK;
}

int rebuild(ls_ctx* c, bool full_scan, cudaStream_t s)
{
    NvtxRange range("ls band rebuild");
    const bool incr = c->band_valid;
    void* cur = c->phi[c->cur];
    const bool incr_mode = c->rebuild_mode == LS_REBUILD_INCREMENTAL ||
                           (c->rebuild_mode == LS_REBUILD_AUTO && c->ntiles >= LS_REBUILD_AUTO_TILES);
    if (incr_mode && !full_scan && c->core_fresh && c->band_valid && !c->full_domain &&
        (c->batched || c->in0().ghost == 0)) {
        RET(rebuild_incr(c, incr, s));
        c->core_fresh = false;
        c->since_rebuild = 0;
        return LS_OK;
    }
    if (full_scan || !c->core_fresh) {
        KL(c, lsk::launch_classify_all(cur, c->core, c->dinst(), c->tinst(), c->in0(), c->ntiles,
                                       c->prec, s));
    } else if (!c->batched && c->in0().ghost) {
        // ghost rows are never active, so the fused tube test of the last
        // step did not see them: test them on their imported values
        const Inst& in = c->in0();
        const long long tpl = (long long)in.tnx * in.tny;
        const size_t row_bytes = (size_t)tpl * lsk::TILE_PTS * c->esize;
        if (in.ghost & 1)
            KL(c, lsk::launch_classify_all(cur, c->core, nullptr, nullptr, in, tpl, c->prec, s));
        if (in.ghost & 2)
            KL(c, lsk::launch_classify_all((char*)cur + (size_t)(in.tnz - 1) * row_bytes,
                                           c->core + (in.tnz - 1) * tpl, nullptr, nullptr, in, tpl,
                                           c->prec, s));
    }
    KL(c, lsk::launch_dilate(c->core, c->act, c->block_counts, c->dinst(), c->tinst(), c->in0(),
                             c->ntiles, c->d_done, c->d_count, c->dilation, s));
    RET(finish_rebuild(c, incr, s));
    c->band_valid = true;
    c->core_fresh = false;
    c->since_rebuild = 0;
    return LS_OK;
}

int full_domain_bound(ls_ctx* c, cudaStream_t s)
{
    if (c->batched) {
        // every tile in the tube: the dilation then marks every tile active
        // and the regular scatter builds the full list, counts and bounds
        CK(cudaMemsetAsync(c->core, 1, c->ntiles, s));
        KL(c, lsk::launch_dilate(c->core, c->act, c->block_counts, c->d_inst, c->d_tile_inst,
                                 c->in0(), c->ntiles, c->d_done, c->d_count, 26, s));
        RET(finish_rebuild(c, false, s));
    } else {
        // every tile counts as active, so a later switch back to a band copies
        // every tile that leaves the active set into the other buffer
        CK(cudaMemsetAsync(c->act, 1, c->ntiles, s));
        KL(c, lsk::launch_full_list(c->list, c->list_info, sign_table(c), const_sign_bits(c),
                                    c->in0(), c->ntiles, c->d_count, c->list_nact, s));
        if (speed_mode(c) == 2)
            KL(c, lsk::launch_max_all(c->tile_maxF, c->ntiles, c->prec, c->d_Mbits, s));
        KL(c, lsk::launch_set_dt(c->d_sc, 1, nullptr, c->in0(), c->dt_mode, c->dt_value, 1,
                                 c->prec, c->d_Mbits, nullptr, c->ntiles, s));
    }
    c->band_valid = true;
    return LS_OK;
}

lsk::StepArgs step_args(ls_ctx* c, bool classify)
{
    lsk::StepArgs a{};
    a.src = c->phi[c->cur];
    a.dst = c->phi[c->cur ^ 1];
    a.F = (speed_mode(c) == 2) ? c->F : nullptr;
    a.list = c->list;
    a.info = c->list_info;
    a.list_inst = c->batched ? c->d_list_inst : nullptr;
    a.count = c->d_count;
    a.sc = c->d_sc;
    a.insts = c->batched ? c->d_inst : nullptr;
    a.core = classify ? c->core : nullptr;
    a.updates = c->d_updates;
    a.status = c->d_status;
    a.in = c->in0();
    a.max_grid = c->full_domain ? (int)(c->ntiles < (1 << 30) ? c->ntiles : (1 << 30)) : 0;
    // copies of the frozen x-faces (plain scheme: no pass between rebuilds
    // writes a tile outside the list), read by the DRAM-bound one-warp
    // kernel; the 4- and 8-point kernels, bound by instruction issue, read
    // every x-face in place (the copies measured no faster there)
    if (c->xface && !c->full_domain && c->scheme == LS_SCHEME_PLAIN && c->step_mode == LS_PLAIN &&
        c->cfg.ppt == 16) {
        a.xface = c->xface;
        a.xface_fill = c->xface_pending ? 1 : 0;
        a.nact = c->list_nact;
    }
    return a;
}

int local_iters(const ls_ctx* c)
{
    if (c->reinit_iters >= 0) return c->reinit_iters;
    return (int)std::ceil(c->halfwidth / c->dtau_in_h - 1e-12);
}

// FP32 copies of the local scheme's thresholds: the branch thresholds are
// rounded outward so that float comparisons decide as the FP64 ones do
lsk::LocalParams local_params(const ls_ctx* c)
{
    const Inst& in = c->insts[0];
    lsk::LocalParams lp{};
    lp.gamma = in.gamma;
    lp.beta = c->beta_in_h * in.h;
    lp.dtau = c->dtau_in_h * in.h;
    float b = (float)lp.beta;
    if ((double)b > lp.beta) b = std::nextafter(b, -INFINITY);
    float g = (float)lp.gamma;
    if ((double)g < lp.gamma) g = std::nextafter(g, INFINITY);
    lp.beta_dn = b;
    lp.gamma_up = g;
    lp.beta_n = (float)lp.beta;
    lp.gamma_n = (float)lp.gamma;
    const double w = lp.gamma - lp.beta;
    lp.inv_w = (float)(1.0 / w);
    lp.lam = (float)c->dtau_in_h;
    lp.dtau_f = (float)lp.dtau;
    return lp;
}

// Profiling: one event pair brackets each run of back-to-back stencil
// launches of one kind (plain / advance, or reinitialisation); any other
// kernel closes the run.  The time per launch is then the run's time over
// its launches (gaps between them included), without an event record
// between every two launches.
int prof_close(ls_ctx* c, cudaStream_t s)
{
    if (!c->ev_open) return LS_OK;
    if (c->ev_skip) {
        c->ev_open = false;
        c->ev_skip = false;
        return LS_OK;
    }
    cudaEvent_t e1 = nullptr;
    CK(take_event(c, &e1));
    CK(cudaEventRecord(e1, s));
    c->ev_pending.push_back({c->ev_open_e0, e1, c->ev_open_kind == 1, c->ev_open_n});
    c->ev_open = false;
    return LS_OK;
}

// a: the launch about to be made; its updates also go to the timed counter
// when its run is timed.  With prof_every = N > 1 one run in N is timed
// (fewer event records between launches, which otherwise cost their overlap).
int prof_before_stencil(ls_ctx* c, int kind, cudaStream_t s, lsk::StepArgs& a)
{
    a.updates_timed = nullptr;
    if (!c->profiling) return LS_OK;
    if (c->ev_open && c->ev_open_kind != kind) RET(prof_close(c, s));
    if (!c->ev_open && (c->prof_runs++ % (unsigned long long)c->prof_every) != 0) {
        c->ev_open = true;
        c->ev_skip = true;
        c->ev_open_kind = kind;
        return LS_OK;
    }
    if (c->ev_skip) return LS_OK;
    a.updates_timed = c->d_updates_timed;
    if (!c->ev_open) {
        if (c->ev_pending.size() >= 4096) RET(drain_events(c));
        CK(take_event(c, &c->ev_open_e0));
        CK(cudaEventRecord(c->ev_open_e0, s));
        c->ev_open = true;
        c->ev_open_kind = kind;
        c->ev_open_n = 0;
    }
    ++c->ev_open_n;
    return LS_OK;
}

bool two_step_ok(const ls_ctx* c)
{
    return c->prec == LS_FP32 && !c->batched && c->scheme == LS_SCHEME_PLAIN &&
           c->step_mode == LS_PLAIN && c->list_nact != nullptr;
}

// the step loop of ls_step (eager, or recorded into a graph by the caller)
int run_steps(ls_ctx* c, int nsteps, double value, int dt_mode, int rebuild_every, cudaStream_t s)
{
    bool dt_pending = true;
    // the previous launch of this call was a plain step over the current
    // list and dt (the next step may read the list before waiting for it)
    bool prev_step = false;
    for (int k = 0; k < nsteps;) {
        bool rebuilt = false;
        if (c->profiling && (!c->band_valid || (rebuild_every > 0 && c->since_rebuild >= rebuild_every) ||
                             (dt_pending && k == 0)))
            RET(prof_close(c, s));
        if (c->full_domain) {
            if (!c->band_valid) {
                RET(full_domain_bound(c, s));
                rebuilt = true;
            }
        } else if (!c->band_valid) {
            RET(rebuild(c, true, s));
            rebuilt = true;
        } else if (rebuild_every > 0 && c->since_rebuild >= rebuild_every) {
            RET(rebuild(c, false, s));
            rebuilt = true;
        }
        if (rebuilt) prev_step = false;
        if (dt_pending && !rebuilt && dt_mode != LS_DT_KEEP) {
            prev_step = false;
            if (c->batched)
                KL(c, lsk::launch_set_dt_batch(c->d_sc, c->n_inst, c->d_inst, dt_mode, value, 0,
                                               c->prec, c->d_Mbits, c->d_inst_count, s));
            else
                KL(c, lsk::launch_set_dt(c->d_sc, 1, nullptr, c->in0(), dt_mode, value, 0, c->prec,
                                         c->d_Mbits, nullptr, 0, s));
        }
        dt_pending = false;
        // two steps per pass (temporal blocking) when configured and both
        // steps fall inside one rebuild period (one dt) with no snapshot after
        // the first of them
        const bool two = c->cfg.spp == 2 && two_step_ok(c) && k + 1 < nsteps &&
                         (rebuild_every == 0 || c->full_domain ||
                          c->since_rebuild + 2 <= rebuild_every) &&
                         !(c->output && (c->step_count + 1) % c->output_every == 0);
        const int adv = two ? 2 : 1;
        // the fused tube test sees the plain step's values; with the learned
        // correction applied afterwards the rebuild classifies again instead
        const bool classify = !c->full_domain && rebuild_every > 0 &&
                              c->since_rebuild + adv >= rebuild_every && c->step_mode == LS_PLAIN;
        if (two) {
            lsk::StepArgs a = step_args(c, classify);
            a.nact = c->list_nact;
            a.updates2 = c->d_updates2;
            RET(prof_before_stencil(c, 0, s, a));
            a.reverse = c->dir;
            KL(c, lsk::launch_step2(a, c->cfg, s));
            prev_step = false;
            c->stencil_launches += 1;
            c->dir ^= 1;
            c->cur ^= 1;
            c->since_rebuild += 2;
            c->core_fresh = classify;
            c->step_count += 2;
            k += 2;
            if (c->output && c->step_count % c->output_every == 0) {
                if (c->profiling) RET(prof_close(c, s));
                RET(ls_engine_output_after_step(c, s));
            }
            continue;
        }
        // plain: one pass; local scheme: the cut-off advance, then the
        // reinitialisation passes (the last one clamps); the fused tube test
        // goes with the last pass of the step
        const bool local = c->scheme == LS_SCHEME_LOCAL;
        const int K = local ? local_iters(c) : 0;
        const int npass = 1 + K;
        for (int p = 0; p < npass; ++p) {
            const bool last = p == npass - 1;
            lsk::StepArgs a = step_args(c, classify && last);
            if (local) {
                a.op = p == 0 ? (K == 0 ? lsk::OP_CUT_CLAMP : lsk::OP_CUT)
                              : (last ? lsk::OP_REINIT_CLAMP : lsk::OP_REINIT);
                a.lp = local_params(c);
                a.nmask = c->nmask;
                a.nact = c->list_nact;
                a.nflag = c->nflag;
                a.breaches = p == 0 ? c->d_breaches : nullptr;
                if (p > 0) {
                    // the reinitialisation passes visit only the tiles that
                    // hold a point of N (compacted after the advance)
                    a.F = nullptr;
                    a.list = c->nl;
                    a.info = c->nl_info;
                    a.count = c->d_ncount;
                    a.nmask = c->nmask2;
                    a.updates = c->d_rupdates;
                }
            }
            RET(prof_before_stencil(c, p > 0 ? 1 : 0, s, a));
            a.reverse = c->dir;
            if (!local && c->full_domain && c->cfg.dense && two_step_ok(c)) {
                a.tile_sgn = sign_table(c);
                KL(c, lsk::launch_dense_step(a, c->cfg, s));
                prev_step = false;
            } else {
                // reinitialisation passes after the first: the previous launch
                // was the pass before, over the same list of N tiles
                a.early = local ? (p >= 2 ? 1 : 0) : (prev_step ? 1 : 0);
                KL(c, lsk::launch_step(a, c->prec, c->cfg, s));
                if (a.xface_fill) c->xface_pending = false;  // this step wrote the copies
                prev_step = !local && c->step_mode != LS_LEARNED;
            }
            ++c->stencil_launches;
            c->dir ^= 1;
            if (c->step_mode == LS_LEARNED) {
                if (c->profiling) RET(prof_close(c, s));
                RET(ls_engine_learned_after_step(c, s));
            }
            c->cur ^= 1;
            if (local && p == 0 && K > 0) {
                if (c->profiling) RET(prof_close(c, s));
                KL(c, lsk::launch_nflag_count(c->nflag, c->d_count, c->block_counts, c->nblocks,
                                              c->d_done + 2, c->d_ncount, s));
                KL(c, lsk::launch_nflag_scatter(c->nflag, c->d_count, c->block_counts, c->list,
                                                c->list_info, c->nmask, c->nl, c->nl_info,
                                                c->nmask2, classify ? c->core : nullptr,
                                                c->nblocks, s));
            }
        }
        c->since_rebuild += 1;
        c->core_fresh = classify;
        c->step_count += 1;
        k += 1;
        if (c->output && c->step_count % c->output_every == 0) {
            if (c->profiling) RET(prof_close(c, s));
            RET(ls_engine_output_after_step(c, s));
            prev_step = false;
        }
    }
    if (c->profiling) RET(prof_close(c, s));
    return LS_OK;
}

SchedState save_state(const ls_ctx* c)
{
    SchedState st;
    st.cur = c->cur;
    st.since_rebuild = c->since_rebuild;
    st.band_valid = c->band_valid;
    st.core_fresh = c->core_fresh;
    st.dir = c->dir;
    st.xface_pending = c->xface_pending;
    return st;
}

void load_state(ls_ctx* c, const SchedState& st)
{
    c->cur = st.cur;
    c->since_rebuild = st.since_rebuild;
    c->band_valid = st.band_valid;
    c->core_fresh = st.core_fresh;
    c->dir = st.dir;
    c->xface_pending = st.xface_pending;
}

cudaStream_t work_stream(ls_ctx* c)
{
    if (c->stream) return c->stream;
    if (!c->own_stream) {
        if (cudaStreamCreate(&c->own_stream) != cudaSuccess) return nullptr;
    }
    return c->own_stream;
}

// ls_step through a cached CUDA graph: the first call with a given starting
// state records the launches, later calls replay them
int run_steps_graph(ls_ctx* c, int nsteps, double value, int dt_mode, int rebuild_every)
{
    cudaStream_t s = work_stream(c);
    if (!s) return cuda_fail(cudaErrorInvalidResourceHandle);
    long long vbits = 0;
    std::memcpy(&vbits, &value, sizeof(vbits));
    const GraphKey key{c->cur, c->since_rebuild, (int)c->band_valid, (int)c->core_fresh,
                       (int)c->full_domain | (c->step_mode << 1) | (c->scheme << 3) |
                           ((int)c->xface_pending << 5),
                       nsteps,
                       rebuild_every, dt_mode, vbits,
                       c->cfg.stages * 16 + c->cfg.ppt + 256 * c->cfg.spp, c->cfg.grid_pct, c->dir};
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
        if (c->graphs.size() >= 16) clear_graphs(c);
        const SchedState before = save_state(c);
        const unsigned long long l0 = c->launches, s0 = c->stencil_launches;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int r = run_steps(c, nsteps, value, dt_mode, rebuild_every, s);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (r != LS_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            load_state(c, before);
            return r != LS_OK ? r : cuda_fail(e);
        }
        GraphEntry ent;
        e = cudaGraphInstantiate(&ent.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            load_state(c, before);
            return cuda_fail(e);
        }
        ent.after = save_state(c);
        ent.launches = c->launches - l0;
        ent.stencil_launches = c->stencil_launches - s0;
        c->launches = l0;
        c->stencil_launches = s0;
        it = c->graphs.emplace(key, ent).first;
    }
    CK(cudaGraphLaunch(it->second.exec, s));
    load_state(c, it->second.after);
    c->launches += it->second.launches;
    c->stencil_launches += it->second.stencil_launches;
    return LS_OK;
}

int make_ctx(int n, const int* nx, const int* ny, const int* nz, const double* h, int precision,
             bool batched, ls_ctx** out)
{
    if (!out) return LS_EINVAL;
    *out = nullptr;
    if (n < 1 || n > 65535 || !nx || !ny || !nz || !h) return LS_EINVAL;
    if (precision != LS_FP32 && precision != LS_FP64) return LS_EINVAL;
    if (batched && precision != LS_FP32) return LS_EINVAL;
    long long total_tiles = 0, total_pts = 0, max_pts = 0;
    for (int i = 0; i < n; ++i) {
        if (nx[i] < 8 || ny[i] < 8 || nz[i] < 8 || nx[i] % 8 || ny[i] % 8 || nz[i] % 8) return LS_EINVAL;
        if (!(h[i] > 0.0) || !std::isfinite(h[i])) return LS_EINVAL;
        const long long pts = (long long)nx[i] * ny[i] * nz[i];
        total_pts += pts;
        total_tiles += pts / lsk::TILE_PTS;
        if (pts > max_pts) max_pts = pts;
    }
    if (total_pts > (1ll << 31)) return LS_EINVAL;
    ls_ctx* c = new (std::nothrow) ls_ctx();
    if (!c) return LS_ENOMEM;
    c->prec = precision;
    c->esize = precision == LS_FP32 ? 4 : 8;
    c->batched = batched;
    c->n_inst = n;
    c->insts.resize(n);
    c->inst_phi_set.assign(n, 0);
    long long base = 0;
    for (int i = 0; i < n; ++i) {
        Inst& in = c->insts[i];
        std::memset(&in, 0, sizeof(in));
        in.nx = nx[i]; in.ny = ny[i]; in.nz = nz[i];
        in.tnx = nx[i] / 8; in.tny = ny[i] / 8; in.tnz = nz[i] / 8;
        in.tile_base = base;
        in.ntiles = (long long)in.tnx * in.tny * in.tnz;
        in.h = h[i];
        in.inv_h = 1.0 / h[i];
        in.pow2h = is_pow2(h[i]) ? 1 : 0;
        in.bc = LS_BC_EXTRAPOLATE;
        base += in.ntiles;
    }
    c->ntiles = total_tiles;
    c->npts = (size_t)total_pts;
    c->max_inst_pts = (size_t)max_pts;
    c->nblocks = (int)((c->ntiles + 255) / 256);
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess && r != cudaSuccess) e = r; };
    A(dalloc(&c->phi[0], grid_bytes(c)));
    A(dalloc(&c->phi[1], grid_bytes(c)));
    A(dalloc(&c->core, c->ntiles));
    // the flag arrays in whole 16-byte chunks (the incremental batch rebuild
    // reads and writes them 16 tiles at a time)
    const long long flag_bytes = (c->ntiles + 15) / 16 * 16;
    A(dalloc(&c->act, flag_bytes));
    A(dalloc(&c->list, c->ntiles * sizeof(int)));
    A(dalloc(&c->list_info, c->ntiles));
    A(dalloc(&c->d_count, sizeof(int)));
    A(dalloc(&c->d_done, 4 * sizeof(unsigned)));
    A(dalloc(&c->d_updates2, sizeof(unsigned long long)));
    if (e == cudaSuccess) e = cudaMemset(c->d_updates2, 0, sizeof(unsigned long long));
    A(dalloc(&c->d_updates_timed, sizeof(unsigned long long)));
    if (e == cudaSuccess) e = cudaMemset(c->d_updates_timed, 0, sizeof(unsigned long long));
    A(dalloc(&c->mark, flag_bytes));
    A(dalloc(&c->d_leave, c->ntiles * sizeof(int)));
    A(dalloc(&c->d_nleave, sizeof(int)));
    if (!batched && precision == LS_FP32) A(dalloc(&c->list_nact, c->ntiles));
    if (!batched && precision == LS_FP32)
        A(dalloc(&c->xface, (size_t)c->ntiles * lsk::XFACE_FLOATS * sizeof(float)));
    if (e == cudaSuccess) e = cudaMemset(c->d_done, 0, 4 * sizeof(unsigned));
    A(dalloc(&c->block_counts, c->nblocks * sizeof(int)));
    A(dalloc(&c->d_sc, sizeof(lsk::StepScalars) * n));
    A(dalloc(&c->d_Mbits, sizeof(unsigned long long) * n));
    A(dalloc(&c->d_updates, sizeof(unsigned long long)));
    A(dalloc(&c->d_status, sizeof(unsigned)));
    A(cudaHostAlloc((void**)&c->h_nonfinite, sizeof(unsigned), cudaHostAllocMapped | cudaHostAllocPortable));
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&c->d_nonfinite, c->h_nonfinite, 0);
    if (batched) {
        A(dalloc(&c->d_inst, sizeof(Inst) * n));
        A(dalloc(&c->d_tile_inst, sizeof(uint16_t) * c->ntiles));
        A(dalloc(&c->d_list_inst, sizeof(uint16_t) * c->ntiles));
        A(dalloc(&c->d_inst_count, sizeof(int) * n));
    }
    if (e == cudaSuccess) {
        A(cudaMemset(c->core, 0, c->ntiles));
        A(cudaMemset(c->act, 0, flag_bytes));
        A(cudaMemset(c->mark, 0, flag_bytes));
        A(cudaMemset(c->d_count, 0, sizeof(int)));
        A(cudaMemset(c->d_sc, 0, sizeof(lsk::StepScalars) * n));
        A(cudaMemset(c->d_Mbits, 0, sizeof(unsigned long long) * n));
        A(cudaMemset(c->d_updates, 0, sizeof(unsigned long long)));
        A(cudaMemset(c->d_status, 0, sizeof(unsigned)));
        if (batched) {
            std::vector<uint16_t> ti((size_t)c->ntiles);
            for (int i = 0; i < n; ++i)
                for (long long t = 0; t < c->insts[i].ntiles; ++t)
                    ti[(size_t)(c->insts[i].tile_base + t)] = (uint16_t)i;
            A(cudaMemcpy(c->d_tile_inst, ti.data(), ti.size() * sizeof(uint16_t),
                         cudaMemcpyHostToDevice));
            A(cudaMemcpy(c->d_inst, c->insts.data(), sizeof(Inst) * n, cudaMemcpyHostToDevice));
            A(cudaMemset(c->d_inst_count, 0, sizeof(int) * n));
        }
        A(cudaDeviceSynchronize());
    }
    if (e != cudaSuccess) {
        free_all(c);
        delete c;
        return cuda_fail(e);
    }
    *out = c;
    return LS_OK;
}

bool all_phi_set(const ls_ctx* c)
{
    for (char f : c->inst_phi_set)
        if (!f) return false;
    return true;
}

int set_phi_inst(ls_ctx* c, int i, const void* src, int on_device)
{
    if (!c || !src || i < 0 || i >= c->n_inst) return LS_EINVAL;
    state_changed(c);
    const Inst& in = c->insts[i];
    c->inst_phi_set[i] = 0;
    RET(pack_from(c, in, src, on_device, region(c, c->phi[c->cur], in)));
    KL(c, lsk::launch_copy(region(c, c->phi[c->cur ^ 1], in), region(c, c->phi[c->cur], in),
                           inst_bytes(c, in), c->stream));
    c->inst_phi_set[i] = 1;
    return LS_OK;
}

int set_speed_inst(ls_ctx* c, int i, const void* src, int on_device)
{
    if (!c || !src || i < 0 || i >= c->n_inst) return LS_EINVAL;
    if (!c->F) CK(dalloc(&c->F, grid_bytes(c)));
    if (!c->tile_maxF) CK(dalloc(&c->tile_maxF, c->ntiles * c->esize));
    if (!c->tile_sgn) CK(dalloc(&c->tile_sgn, c->ntiles));
    state_changed(c);
    Inst& in = c->insts[i];
    in.speed_mode = 0;
    RET(pack_from(c, in, src, on_device, region(c, c->F, in)));
    KL(c, lsk::launch_tile_speed(region(c, c->F, in),
                                 (char*)c->tile_maxF + (size_t)in.tile_base * c->esize,
                                 c->tile_sgn + in.tile_base, in.ntiles, c->prec, c->stream));
    in.speed_mode = 2;
    return upload_insts(c);
}

int set_speed_const_inst(ls_ctx* c, int i, double F)
{
    if (!c || i < 0 || i >= c->n_inst) return LS_EINVAL;
    if (!std::isfinite(F)) return LS_ENONFINITE;
    state_changed(c);
    c->insts[i].Fc = F;
    c->insts[i].speed_mode = 1;
    return upload_insts(c);
}

int get_phi_inst(ls_ctx* c, int i, void* dst, int on_device)
{
    if (!c || !dst || i < 0 || i >= c->n_inst) return LS_EINVAL;
    if (!c->inst_phi_set[i]) return LS_ESTATE;
    const Inst& in = c->insts[i];
    const void* srcb = region(c, c->phi[c->cur], in);
    if (on_device) {
        if (!aligned16(dst)) return LS_EINVAL;
        KL(c, lsk::launch_unpack(srcb, dst, in, c->prec, c->stream));
    } else {
        RET(ensure_staging(c));
        KL(c, lsk::launch_unpack(srcb, c->staging, in, c->prec, c->stream));
        CK(cudaMemcpyAsync(dst, c->staging, inst_bytes(c, in), cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return LS_OK;
}

// copy the (global) active list to the host
int fetch_list(ls_ctx* c, std::vector<int>& ids)
{
    int cnt = 0;
    CK(cudaMemcpyAsync(&cnt, c->d_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    ids.resize((size_t)cnt);
    if (cnt > 0) {
        CK(cudaMemcpyAsync(ids.data(), c->list, sizeof(int) * cnt, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return LS_OK;
}

}  // namespace

int ls_engine_cuda_fail(cudaError_t e) { return cuda_fail(e); }

int ls_engine_pack(ls_ctx* c, const Inst& in, const void* src, int on_device, void* dst)
{
    return pack_from(c, in, src, on_device, dst);
}

extern "C" {

const char* ls_strerror(int st)
{
    switch (st) {
    case LS_OK: return "ok";
    case LS_EINVAL: return "invalid argument";
    case LS_ENOMEM: return "out of device or host memory";
    case LS_ECUDA: return "CUDA error";
    case LS_ETIMEOUT: return "bounded device wait timed out";
    case LS_ENONFINITE: return "non-finite value in input";
    case LS_ESTATE: return "call not valid in the current state";
    case LS_EIO: return "output file could not be written";
    default: return "unknown status";
    }
}

int ls_last_cuda_error(void) { return g_last_cuda_error; }

int ls_create(int nx, int ny, int nz, double h, int precision, ls_ctx** out)
{
    return make_ctx(1, &nx, &ny, &nz, &h, precision, false, out);
}

int ls_batch_create(int n, const int* nx, const int* ny, const int* nz, const double* h,
                    int precision, ls_ctx** out)
{
    return make_ctx(n, nx, ny, nz, h, precision, true, out);
}

int ls_batch_size(ls_ctx* c, int* n)
{
    if (!c || !n) return LS_EINVAL;
    *n = c->n_inst;
    return LS_OK;
}

int ls_destroy(ls_ctx* c)
{
    if (!c) return LS_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    free_all(c);
    delete c;
    return LS_OK;
}

int ls_set_stream(ls_ctx* c, void* stream)
{
    if (!c) return LS_EINVAL;
    c->stream = (cudaStream_t)stream;
    clear_graphs(c);
    return LS_OK;
}

int ls_set_bc(ls_ctx* c, int bc)
{
    if (!c || (bc != LS_BC_EXTRAPOLATE && bc != LS_BC_NEUMANN)) return LS_EINVAL;
    for (Inst& in : c->insts) in.bc = bc;
    clear_graphs(c);
    return upload_insts(c);
}

int ls_set_phi(ls_ctx* c, const void* src, int on_device)
{
    if (!c || c->n_inst != 1) return LS_EINVAL;
    return set_phi_inst(c, 0, src, on_device);
}

int ls_inst_set_phi(ls_ctx* c, int i, const void* src, int on_device)
{
    return set_phi_inst(c, i, src, on_device);
}

int ls_set_speed(ls_ctx* c, const void* src, int on_device)
{
    if (!c || c->n_inst != 1) return LS_EINVAL;
    return set_speed_inst(c, 0, src, on_device);
}

int ls_inst_set_speed(ls_ctx* c, int i, const void* src, int on_device)
{
    return set_speed_inst(c, i, src, on_device);
}

int ls_set_speed_const(ls_ctx* c, double F)
{
    if (!c) return LS_EINVAL;
    for (int i = 0; i < c->n_inst; ++i) RET(set_speed_const_inst(c, i, F));
    return LS_OK;
}

int ls_inst_set_speed_const(ls_ctx* c, int i, double F) { return set_speed_const_inst(c, i, F); }

int ls_set_full_domain(ls_ctx* c, int on)
{
    if (!c) return LS_EINVAL;
    c->full_domain = on != 0;
    state_changed(c);
    return LS_OK;
}

int ls_set_graphs(ls_ctx* c, int on)
{
    if (!c) return LS_EINVAL;
    c->use_graphs = on != 0;
    if (!c->use_graphs) clear_graphs(c);
    return LS_OK;
}

int ls_band_rebuild(ls_ctx* c, double halfwidth, long long* n_active)
{
    if (!c) return LS_EINVAL;
    if (!(halfwidth > 0.0) || !std::isfinite(halfwidth)) return LS_EINVAL;
    if (!all_phi_set(c)) return LS_ESTATE;
    c->halfwidth = halfwidth;
    c->have_halfwidth = true;
    for (Inst& in : c->insts) in.gamma = halfwidth * in.h;
    clear_graphs(c);
    RET(upload_insts(c));
    RET(rebuild(c, true, c->stream));
    if (n_active) {
        int n = 0;
        CK(cudaMemcpyAsync(&n, c->d_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        *n_active = n;
    }
    return LS_OK;
}

// ---- slab split support -------------------------------------------------

int ls_set_ghost_rows(ls_ctx* c, int lo, int hi)
{
    if (!c || c->batched || (lo != 0 && lo != 1) || (hi != 0 && hi != 1)) return LS_EINVAL;
    Inst& in = c->in0();
    if (in.tnz < 1 + lo + hi) return LS_EINVAL;
    in.ghost = lo | (hi << 1);
    state_changed(c);
    return LS_OK;
}

int ls_band_refresh(ls_ctx* c, double* M, long long* n_active)
{
    if (!c || c->batched) return LS_EINVAL;
    if (!all_phi_set(c) || speed_mode(c) == 0) return LS_ESTATE;
    if (!c->have_halfwidth || c->full_domain) return LS_ESTATE;
    clear_graphs(c);
    // the rebuild ls_step would make now: from the tube test fused into the
    // last step when that step made one, else from a scan of every tile
    RET(rebuild(c, !c->band_valid, c->stream));
    if (!M && !n_active) return LS_OK;  // nothing to read back: no synchronisation
    lsk::StepScalars sc;
    int n = 0;
    CK(cudaMemcpyAsync(&sc, c->d_sc, sizeof(sc), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&n, c->d_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (M) *M = sc.M;
    if (n_active) *n_active = n;
    return LS_OK;
}

int ls_band_speed_bound(ls_ctx* c, double* dst, int on_device)
{
    if (!c || c->batched || !dst) return LS_EINVAL;
    if (!c->band_valid) return LS_ESTATE;
    // StepScalars::M is the first member
    const double* M = &c->d_sc[0].M;
    if (on_device) {
        CK(cudaMemcpyAsync(dst, M, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    } else {
        CK(cudaMemcpyAsync(dst, M, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return LS_OK;
}

int ls_set_dt_from_bound(ls_ctx* c, const double* M_device, double cfl)
{
    if (!c || c->batched || !M_device || !(cfl > 0.0) || !std::isfinite(cfl)) return LS_EINVAL;
    if (!c->band_valid) return LS_ESTATE;
    KL(c, lsk::launch_set_dt_from(c->d_sc, M_device, c->in0(), cfl, c->prec, c->stream));
    return LS_OK;
}

int ls_band_row_counts(ls_ctx* c, long long* counts, int nrows)
{
    if (!c || c->batched || !counts) return LS_EINVAL;
    const Inst& in = c->in0();
    if (nrows != in.tnz) return LS_EINVAL;
    if (!c->band_valid) return LS_ESTATE;
    if (!c->d_rowcnt) CK(cudaMalloc(&c->d_rowcnt, sizeof(int) * (size_t)in.tnz));
    CK(cudaMemsetAsync(c->d_rowcnt, 0, sizeof(int) * (size_t)in.tnz, c->stream));
    KL(c, lsk::launch_row_counts(c->list, c->d_count, in.tnx * in.tny, c->d_rowcnt, in.tnz, c->stream));
    std::vector<int> h((size_t)in.tnz);
    CK(cudaMemcpyAsync(h.data(), c->d_rowcnt, sizeof(int) * h.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < in.tnz; ++i) counts[i] = h[(size_t)i];
    return LS_OK;
}

// copies between the current phi buffer's tile rows [row0, row0 + nrows) and
// a packed buffer: plane < 0: whole rows (tile after tile, 512 values each,
// the bricked order); plane 0..7: that z-plane of every tile (64 values per
// tile, tile after tile)
static int tile_rows_copy(ls_ctx* c, int row0, int nrows, int plane, void* buf, int on_device,
                          bool to_ctx)
{
    const Inst& in = c->in0();
    const size_t tpl = (size_t)in.tnx * in.tny;
    const size_t es = c->esize;
    char* base = (char*)c->phi[c->cur] + (size_t)row0 * tpl * lsk::TILE_PTS * es;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice
                                          : (to_ctx ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
    if (plane < 0) {
        const size_t bytes = (size_t)nrows * tpl * lsk::TILE_PTS * es;
        if (to_ctx) CK(cudaMemcpyAsync(base, buf, bytes, kind, c->stream));
        else CK(cudaMemcpyAsync(buf, base, bytes, kind, c->stream));
    } else if (on_device) {
        // one z-plane (64 values) per tile: a copy kernel (a strided
        // device-to-device cudaMemcpy2D of 256-byte rows is several times slower)
        const long long words = 64 * (long long)es / 4, pitch = lsk::TILE_PTS * (long long)es / 4;
        char* p = base + (size_t)plane * 64 * es;
        if (to_ctx) KL(c, lsk::launch_chunk_copy(buf, words, p, pitch, (int)words, (long long)nrows * tpl, c->stream));
        else KL(c, lsk::launch_chunk_copy(p, pitch, buf, words, (int)words, (long long)nrows * tpl, c->stream));
    } else {
        const size_t w = 64 * es, pitch = lsk::TILE_PTS * es, rows = (size_t)nrows * tpl;
        char* p = base + (size_t)plane * w;
        if (to_ctx) CK(cudaMemcpy2DAsync(p, pitch, buf, w, w, rows, kind, c->stream));
        else CK(cudaMemcpy2DAsync(buf, w, p, pitch, w, rows, kind, c->stream));
    }
    if (!on_device) CK(cudaStreamSynchronize(c->stream));
    return LS_OK;
}

int ls_get_tile_rows(ls_ctx* c, int row0, int nrows, int plane, void* dst, int on_device)
{
    if (!c || c->batched || !dst || plane < -1 || plane > 7) return LS_EINVAL;
    const Inst& in = c->in0();
    if (row0 < 0 || nrows < 1 || row0 + nrows > in.tnz) return LS_EINVAL;
    if (!all_phi_set(c)) return LS_ESTATE;
    return tile_rows_copy(c, row0, nrows, plane, dst, on_device, false);
}

int ls_copy_ghost_row(const ls_ctx* src, int src_row, ls_ctx* c, int row, int plane)
{
    if (!src || !c || src->batched || c->batched || plane < -1 || plane > 7) return LS_EINVAL;
    const Inst& si = src->insts[0];
    const Inst& in = c->in0();
    if (src->prec != c->prec || si.tnx != in.tnx || si.tny != in.tny) return LS_EINVAL;
    if (src_row < 0 || src_row >= si.tnz) return LS_EINVAL;
    const bool lo = (in.ghost & 1) && row == 0;
    const bool hi = (in.ghost & 2) && row == in.tnz - 1;
    if (!lo && !hi) return LS_EINVAL;  // only a ghost row takes a neighbour's values
    if (!src->inst_phi_set[0] || !all_phi_set(c)) return LS_ESTATE;
    clear_graphs(c);
    const size_t tpl = (size_t)in.tnx * in.tny, es = c->esize;
    const char* sb = (const char*)src->phi[src->cur] + (size_t)src_row * tpl * lsk::TILE_PTS * es;
    char* db = (char*)c->phi[c->cur] + (size_t)row * tpl * lsk::TILE_PTS * es;
    if (plane < 0) {
        CK(cudaMemcpyAsync(db, sb, tpl * lsk::TILE_PTS * es, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        const long long words = 64 * (long long)es / 4, pitch = lsk::TILE_PTS * (long long)es / 4;
        KL(c, lsk::launch_chunk_copy(sb + (size_t)plane * 64 * es, pitch, db + (size_t)plane * 64 * es,
                                     pitch, (int)words, (long long)tpl, c->stream));
    }
    return LS_OK;
}

int ls_set_tile_rows(ls_ctx* c, int row0, int nrows, int plane, const void* src, int on_device)
{
    if (!c || c->batched || !src || plane < -1 || plane > 7 || nrows != 1) return LS_EINVAL;
    const Inst& in = c->in0();
    const bool lo = (in.ghost & 1) && row0 == 0;
    const bool hi = (in.ghost & 2) && row0 == in.tnz - 1;
    if (!lo && !hi) return LS_EINVAL;  // only a ghost row takes a neighbour's values
    if (!all_phi_set(c)) return LS_ESTATE;
    clear_graphs(c);
    return tile_rows_copy(c, row0, nrows, plane, const_cast<void*>(src), on_device, true);
}

int ls_step(ls_ctx* c, int nsteps, double value, int dt_mode, int rebuild_every, double* last_dt)
{
    if (!c) return LS_EINVAL;
    if (nsteps < 0 || rebuild_every < 0) return LS_EINVAL;
    if (dt_mode != LS_DT_FIXED && dt_mode != LS_DT_CFL && dt_mode != LS_DT_KEEP) return LS_EINVAL;
    if (dt_mode != LS_DT_KEEP && (!(value > 0.0) || !std::isfinite(value))) return LS_EINVAL;
    if (!all_phi_set(c) || speed_mode(c) == 0) return LS_ESTATE;
    if (!c->full_domain && !c->have_halfwidth) return LS_ESTATE;
    if (c->scheme == LS_SCHEME_LOCAL && (!c->have_halfwidth || !(c->beta_in_h < c->halfwidth)))
        return LS_ESTATE;
    if (dt_mode == LS_DT_KEEP) {
        // the dt on the device stays; every rebuild is the caller's
        // (ls_band_refresh), so none may fall due inside this call
        if (c->batched || c->full_domain || !c->band_valid || c->step_mode != LS_PLAIN)
            return LS_ESTATE;
        if (rebuild_every > 0 && c->since_rebuild + nsteps > rebuild_every) return LS_ESTATE;
    } else {
        c->dt_mode = dt_mode;
        c->dt_value = value;
    }
    NvtxRange range("ls_step");
    if (nsteps > 0) {
        if (c->use_graphs && !c->profiling && !c->output)
            RET(run_steps_graph(c, nsteps, value, dt_mode, rebuild_every));
        else RET(run_steps(c, nsteps, value, dt_mode, rebuild_every, c->stream));
    }
    if (last_dt) {
        lsk::StepScalars sc;
        CK(cudaMemcpyAsync(&sc, c->d_sc, sizeof(sc), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        *last_dt = sc.dt;
    }
    return LS_OK;
}

int ls_inst_last_dt(ls_ctx* c, int i, double* dt)
{
    if (!c || !dt || i < 0 || i >= c->n_inst) return LS_EINVAL;
    lsk::StepScalars sc;
    CK(cudaMemcpyAsync(&sc, c->d_sc + i, sizeof(sc), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *dt = sc.dt;
    return LS_OK;
}

int ls_autotune(ls_ctx* c, int reps, int* stages_out, int* grid_pct_out, int* ppt_out)
{
    if (!c || reps < 1) return LS_EINVAL;
    if (!c->band_valid) return LS_ESTATE;
    cudaStream_t s = c->stream;
    if (c->prec == LS_FP32) {
        const int stages[] = {2, 3, 4, 6};
        const int pcts[] = {50, 75, 100};
        const int ppts[] = {4, 8, 16};
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        float best = 1e30f;
        lsk::StepConfig best_cfg = c->cfg;
        lsk::StepArgs a = step_args(c, false);
        a.updates = nullptr;  // probes write the other buffer only; the state is unchanged
        for (int ppt : ppts)
        for (int st : stages) {
            for (int pct : pcts) {
                lsk::StepConfig cfg;
                cfg.stages = st;
                cfg.grid_pct = pct;
                cfg.ppt = ppt;
                KL(c, lsk::launch_step(a, c->prec, cfg, s));
                CK(cudaEventRecord(e0, s));
                for (int r = 0; r < reps; ++r) KL(c, lsk::launch_step(a, c->prec, cfg, s));
                CK(cudaEventRecord(e1, s));
                CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) {
                    best = ms;
                    best_cfg = cfg;
                }
            }
        }
        // two steps per pass: the time of one pass counts for two steps
        best_cfg.spp = 1;
        if (two_step_ok(c)) {
            lsk::StepArgs a2 = step_args(c, false);
            a2.updates = nullptr;
            a2.nact = c->list_nact;
            for (int pct : pcts) {
                lsk::StepConfig cfg = best_cfg;
                cfg.spp = 2;
                cfg.grid_pct2 = pct;
                KL(c, lsk::launch_step2(a2, cfg, s));
                CK(cudaEventRecord(e0, s));
                for (int r = 0; r < reps; ++r) KL(c, lsk::launch_step2(a2, cfg, s));
                CK(cudaEventRecord(e1, s));
                CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                if (0.5f * ms < best) {
                    best = 0.5f * ms;
                    best_cfg = cfg;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c->cfg = best_cfg;
        clear_graphs(c);
    }
    if (stages_out) *stages_out = c->cfg.stages;
    if (grid_pct_out) *grid_pct_out = c->cfg.grid_pct;
    if (ppt_out) *ppt_out = c->cfg.ppt;
    return LS_OK;
}

int ls_set_dense_kernel(ls_ctx* c, int on)
{
    if (!c) return LS_EINVAL;
    c->cfg.dense = on != 0;
    clear_graphs(c);
    return LS_OK;
}

int ls_set_steps_per_pass(ls_ctx* c, int steps)
{
    if (!c || (steps != 1 && steps != 2)) return LS_EINVAL;
    c->cfg.spp = steps;
    clear_graphs(c);
    return LS_OK;
}

int ls_get_steps_per_pass(ls_ctx* c, int* steps)
{
    if (!c || !steps) return LS_EINVAL;
    *steps = c->cfg.spp;
    return LS_OK;
}

int ls_set_step_config(ls_ctx* c, int stages, int grid_pct, int ppt)
{
    if (!c || (stages != 2 && stages != 3 && stages != 4 && stages != 6) || grid_pct < 1 || grid_pct > 100 ||
        (ppt != 4 && ppt != 8 && ppt != 16))
        return LS_EINVAL;
    c->cfg.stages = stages;
    c->cfg.grid_pct = grid_pct;
    c->cfg.ppt = ppt;
    clear_graphs(c);
    return LS_OK;
}

int ls_snapshot(ls_ctx* c)
{
    if (!c) return LS_EINVAL;
    if (!all_phi_set(c)) return LS_ESTATE;
    if (!c->snapshot) CK(dalloc(&c->snapshot, grid_bytes(c)));
    CK(cudaMemcpyAsync(c->snapshot, c->phi[c->cur], grid_bytes(c), cudaMemcpyDeviceToDevice,
                       c->stream));
    return LS_OK;
}

int ls_restore(ls_ctx* c)
{
    if (!c) return LS_EINVAL;
    if (!c->snapshot) return LS_ESTATE;
    state_changed(c);
    // one read of the snapshot, both buffers written (16-byte multiples:
    // grids are whole 8^3 tiles)
    KL(c, lsk::launch_copy(c->phi[0], c->snapshot, grid_bytes(c), c->stream, c->phi[1]));
    c->cur = 0;
    return LS_OK;
}

static int upload_params(ls_ctx* c, const double* params, int n, double** dev)
{
    static_assert(sizeof(double) == 8, "double");
    if (n > c->init_params_cap) {
        if (c->init_params) cudaFree(c->init_params);
        c->init_params = nullptr;
        c->init_params_cap = 0;
        CK(cudaMalloc(&c->init_params, sizeof(double) * n));
        c->init_params_cap = n;
    }
    CK(cudaMemcpyAsync(c->init_params, params, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));  // params is caller memory: copy before returning
    *dev = c->init_params;
    return LS_OK;
}

static int shape_params_ok(int kind, const double* p, int n)
{
    if (!p || n < 1) return 0;
    if (kind == LS_SHAPE_SPHERES) return n >= 1 && p[0] >= 1 && n == 1 + 4 * (int)p[0];
    if (kind == LS_SHAPE_TORUS) return n == 8;
    if (kind == LS_SHAPE_SH) {
        if (n < 6) return 0;
        const int lmax = (int)p[5];
        if (lmax < 1 || lmax > 16) return 0;
        const int modes = (lmax + 1) * (lmax + 1) - 1;
        return n == 6 + modes;
    }
    return 0;
}

static int speed_params_ok(int kind, const double* p, int n)
{
    if (kind == LS_SPEED_SINUSOID || kind == LS_SPEED_COSCOS) return 1;
    if (kind == LS_SPEED_FOURIER) return p && n >= 1 && p[0] >= 1 && n == 1 + 5 * (int)p[0];
    return 0;
}

int ls_inst_init_phi(ls_ctx* c, int i, int shape, const double* params, int nparams)
{
    if (!c || i < 0 || i >= c->n_inst || !shape_params_ok(shape, params, nparams)) return LS_EINVAL;
    double* dp = nullptr;
    RET(upload_params(c, params, nparams, &dp));
    state_changed(c);
    const Inst& in = c->insts[i];
    KL(c, lsk::launch_init_field(region(c, c->phi[c->cur], in), region(c, c->phi[c->cur ^ 1], in), in,
                                 c->prec, 0, shape, dp, c->stream));
    c->inst_phi_set[i] = 1;
    return LS_OK;
}

int ls_init_phi(ls_ctx* c, int shape, const double* params, int nparams)
{
    if (!c || c->n_inst != 1) return LS_EINVAL;
    return ls_inst_init_phi(c, 0, shape, params, nparams);
}

int ls_inst_init_speed(ls_ctx* c, int i, int kind, const double* params, int nparams)
{
    if (!c || i < 0 || i >= c->n_inst || !speed_params_ok(kind, params, nparams)) return LS_EINVAL;
    if (!c->F) CK(dalloc(&c->F, grid_bytes(c)));
    if (!c->tile_maxF) CK(dalloc(&c->tile_maxF, c->ntiles * c->esize));
    if (!c->tile_sgn) CK(dalloc(&c->tile_sgn, c->ntiles));
    double* dp = nullptr;
    static const double none = 0.0;
    RET(upload_params(c, params ? params : &none, params ? nparams : 1, &dp));
    state_changed(c);
    Inst& in = c->insts[i];
    KL(c, lsk::launch_init_field(region(c, c->F, in), nullptr, in, c->prec, 1, kind, dp, c->stream));
    KL(c, lsk::launch_tile_speed(region(c, c->F, in), (char*)c->tile_maxF + (size_t)in.tile_base * c->esize,
                                 c->tile_sgn + in.tile_base, in.ntiles, c->prec, c->stream));
    in.speed_mode = 2;
    return upload_insts(c);
}

int ls_init_speed(ls_ctx* c, int kind, const double* params, int nparams)
{
    if (!c || c->n_inst != 1) return LS_EINVAL;
    return ls_inst_init_speed(c, 0, kind, params, nparams);
}

int ls_selftest_bounded_wait(unsigned* status, long long polls, void* stream)
{
    if (!status || polls < 1) return LS_EINVAL;
    CK(lsk::launch_selftest_wait(status, polls, (cudaStream_t)stream));
    return LS_OK;
}

int ls_get_phi(ls_ctx* c, void* dst, int on_device)
{
    if (!c || c->n_inst != 1) return LS_EINVAL;
    return get_phi_inst(c, 0, dst, on_device);
}

int ls_inst_get_phi(ls_ctx* c, int i, void* dst, int on_device)
{
    return get_phi_inst(c, i, dst, on_device);
}

int ls_get_speed(ls_ctx* c, void* dst, int on_device)
{
    if (!c || !dst || c->n_inst != 1) return LS_EINVAL;
    const Inst& in = c->insts[0];
    if (!c->F || in.speed_mode != 2) return LS_ESTATE;
    const void* srcb = region(c, c->F, in);
    if (on_device) {
        if (!aligned16(dst)) return LS_EINVAL;
        KL(c, lsk::launch_unpack(srcb, dst, in, c->prec, c->stream));
    } else {
        RET(ensure_staging(c));
        KL(c, lsk::launch_unpack(srcb, c->staging, in, c->prec, c->stream));
        CK(cudaMemcpyAsync(dst, c->staging, inst_bytes(c, in), cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return LS_OK;
}

// ---- stream-ordered host input/output ----
static int hostio(ls_ctx* c, lsk::HostIO** out)
{
    if (!c->hio) {
        lsk::HostIO* H = new lsk::HostIO();
        c->hio = H;  // freed with the context even if a step below fails
        CK(cudaStreamCreateWithFlags(&H->h2d, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&H->d2h, cudaStreamNonBlocking));
        for (cudaEvent_t* e : {&H->staged, &H->consumed, &H->unpacked, &H->drained})
            CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        // recorded once so that the first waits on them pass
        CK(cudaEventRecord(H->consumed, c->stream));
        CK(cudaEventRecord(H->drained, H->d2h));
    }
    *out = c->hio;
    return LS_OK;
}

int ls_stage_inputs(ls_ctx* c, const void* phi_host, const void* speed_host)
{
    if (!c || c->n_inst != 1 || !phi_host) return LS_EINVAL;
    lsk::HostIO* H = nullptr;
    RET(hostio(c, &H));
    if (H->have_phi) return LS_ESTATE;  // the staged inputs were not loaded yet
    const size_t bytes = grid_bytes(c);
    if (!H->in_phi) CK(dalloc(&H->in_phi, bytes));
    if (speed_host && !H->in_F) CK(dalloc(&H->in_F, bytes));
    // the previous ls_load_staged must have read the buffers
    CK(cudaStreamWaitEvent(H->h2d, H->consumed, 0));
    CK(cudaMemcpyAsync(H->in_phi, phi_host, bytes, cudaMemcpyHostToDevice, H->h2d));
    if (speed_host) CK(cudaMemcpyAsync(H->in_F, speed_host, bytes, cudaMemcpyHostToDevice, H->h2d));
    CK(cudaEventRecord(H->staged, H->h2d));
    H->have_phi = true;
    H->have_F = speed_host != nullptr;
    return LS_OK;
}

int ls_load_staged(ls_ctx* c)
{
    if (!c || c->n_inst != 1) return LS_EINVAL;
    lsk::HostIO* H = c->hio;
    if (!H || !H->have_phi) return LS_ESTATE;
    CK(cudaStreamWaitEvent(c->stream, H->staged, 0));
    H->have_phi = false;
    const bool F = H->have_F;
    H->have_F = false;
    int st = set_phi_inst(c, 0, H->in_phi, 1);
    if (st == LS_OK && F) st = set_speed_inst(c, 0, H->in_F, 1);
    CK(cudaEventRecord(H->consumed, c->stream));
    return st;
}

int ls_get_phi_async(ls_ctx* c, void* host_dst)
{
    if (!c || c->n_inst != 1 || !host_dst) return LS_EINVAL;
    if (!c->inst_phi_set[0]) return LS_ESTATE;
    lsk::HostIO* H = nullptr;
    RET(hostio(c, &H));
    const size_t bytes = grid_bytes(c);
    if (!H->out) CK(dalloc(&H->out, bytes));
    // the previous read-back must have left the staging buffer
    CK(cudaStreamWaitEvent(c->stream, H->drained, 0));
    KL(c, lsk::launch_unpack(c->phi[c->cur], H->out, c->insts[0], c->prec, c->stream));
    CK(cudaEventRecord(H->unpacked, c->stream));
    CK(cudaStreamWaitEvent(H->d2h, H->unpacked, 0));
    CK(cudaMemcpyAsync(host_dst, H->out, bytes, cudaMemcpyDeviceToHost, H->d2h));
    CK(cudaEventRecord(H->drained, H->d2h));
    return LS_OK;
}

int ls_wait_host(ls_ctx* c)
{
    if (!c) return LS_EINVAL;
    if (!c->hio) return LS_OK;
    CK(cudaStreamSynchronize(c->hio->h2d));
    CK(cudaStreamSynchronize(c->hio->d2h));
    return LS_OK;
}

int ls_get_active_tiles(ls_ctx* c, int* dst, long long cap, long long* n)
{
    if (!c || !n || cap < 0 || (cap > 0 && !dst)) return LS_EINVAL;
    if (!c->band_valid) return LS_ESTATE;
    std::vector<int> ids;
    RET(fetch_list(c, ids));
    *n = (long long)ids.size();
    const long long k = cap < *n ? cap : *n;
    if (k > 0) std::memcpy(dst, ids.data(), sizeof(int) * k);
    return LS_OK;
}

int ls_inst_get_active_tiles(ls_ctx* c, int i, int* dst, long long cap, long long* n)
{
    if (!c || !n || cap < 0 || (cap > 0 && !dst) || i < 0 || i >= c->n_inst) return LS_EINVAL;
    if (!c->band_valid) return LS_ESTATE;
    std::vector<int> ids;
    RET(fetch_list(c, ids));
    const Inst& in = c->insts[i];
    long long k = 0;
    for (int t : ids) {
        if (t < in.tile_base || t >= in.tile_base + in.ntiles) continue;
        if (k < cap) dst[k] = (int)(t - in.tile_base);
        ++k;
    }
    *n = k;
    return LS_OK;
}

int ls_get_updates(ls_ctx* c, unsigned long long* n)
{
    if (!c || !n) return LS_EINVAL;
    CK(cudaMemcpyAsync(n, c->d_updates, sizeof(*n), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LS_OK;
}

int ls_profile_enable(ls_ctx* c, int on)
{
    if (!c) return LS_EINVAL;
    if (on < 0) return LS_EINVAL;
    if (c->ev_open) RET(prof_close(c, c->stream));
    c->profiling = on != 0;
    c->prof_every = on > 0 ? on : 1;
    c->prof_runs = 0;
    return LS_OK;
}

int ls_get_profile(ls_ctx* c, ls_profile* out)
{
    if (!c || !out) return LS_EINVAL;
    RET(drain_events(c));
    out->kernel_launches = c->launches;
    out->stencil_launches = c->stencil_launches;
    out->stencil_ms = c->stencil_ms;
    out->stencil_timed = c->stencil_timed;
    out->reinit_ms = c->reinit_ms;
    out->reinit_timed = c->reinit_timed;
    out->reinit_updates = 0;
    CK(cudaMemcpyAsync(&out->two_step_points, c->d_updates2, sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->d_rupdates) {
        CK(cudaMemcpyAsync(&out->reinit_updates, c->d_rupdates, sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    CK(cudaMemcpyAsync(&out->stencil_updates, c->d_updates_timed, sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LS_OK;
}

int ls_reset_profile(ls_ctx* c)
{
    if (!c) return LS_EINVAL;
    RET(drain_events(c));
    c->launches = 0;
    c->stencil_launches = 0;
    c->stencil_ms = 0.0;
    c->stencil_timed = 0;
    c->reinit_ms = 0.0;
    c->reinit_timed = 0;
    CK(cudaMemsetAsync(c->d_updates_timed, 0, sizeof(unsigned long long), c->stream));
    return LS_OK;
}

int ls_set_scheme(ls_ctx* c, int scheme, double beta_in_h, int reinit_iters, double dtau_in_h)
{
    if (!c) return LS_EINVAL;
    if (scheme == LS_SCHEME_PLAIN) {
        c->scheme = LS_SCHEME_PLAIN;
        clear_graphs(c);
        return LS_OK;
    }
    if (scheme != LS_SCHEME_LOCAL || c->batched) return LS_EINVAL;
    if (!(beta_in_h > 0.0) || !std::isfinite(beta_in_h)) return LS_EINVAL;
    if (!(dtau_in_h > 0.0) || !std::isfinite(dtau_in_h)) return LS_EINVAL;
    if (reinit_iters < -1) return LS_EINVAL;
    if (c->step_mode != LS_PLAIN) return LS_ESTATE;
    if (!c->nmask) CK(dalloc(&c->nmask, (size_t)c->ntiles * 16 * sizeof(uint32_t)));
    if (!c->nmask2) CK(dalloc(&c->nmask2, (size_t)c->ntiles * 16 * sizeof(uint32_t)));
    if (!c->nflag) CK(dalloc(&c->nflag, (size_t)c->ntiles));
    if (!c->nl) CK(dalloc(&c->nl, (size_t)c->ntiles * sizeof(int)));
    if (!c->nl_info) CK(dalloc(&c->nl_info, (size_t)c->ntiles));
    if (!c->d_ncount) CK(dalloc(&c->d_ncount, sizeof(int)));
    if (!c->d_rupdates) {
        CK(dalloc(&c->d_rupdates, sizeof(unsigned long long)));
        CK(cudaMemsetAsync(c->d_rupdates, 0, sizeof(unsigned long long), c->stream));
    }
    if (!c->list_nact) {
        CK(dalloc(&c->list_nact, (size_t)c->ntiles));
        state_changed(c);  // the next rebuild writes the neighbour bits
    }
    if (!c->d_breaches) CK(dalloc(&c->d_breaches, sizeof(unsigned long long)));
    CK(cudaMemsetAsync(c->d_breaches, 0, sizeof(unsigned long long), c->stream));
    c->scheme = LS_SCHEME_LOCAL;
    c->beta_in_h = beta_in_h;
    c->reinit_iters = reinit_iters;
    c->dtau_in_h = dtau_in_h;
    clear_graphs(c);
    return LS_OK;
}

int ls_set_rebuild_mode(ls_ctx* c, int mode)
{
    if (!c || (mode != LS_REBUILD_AUTO && mode != LS_REBUILD_FULL && mode != LS_REBUILD_INCREMENTAL))
        return LS_EINVAL;
    c->rebuild_mode = mode;
    clear_graphs(c);
    return LS_OK;
}

int ls_set_dilation(ls_ctx* c, int neighbours)
{
    if (!c || (neighbours != 6 && neighbours != 26)) return LS_EINVAL;
    c->dilation = neighbours;
    state_changed(c);
    return LS_OK;
}

int ls_band_breaches(ls_ctx* c, unsigned long long* n)
{
    if (!c || !n) return LS_EINVAL;
    *n = 0;
    if (!c->d_breaches) return LS_OK;
    CK(cudaMemcpyAsync(n, c->d_breaches, sizeof(*n), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LS_OK;
}

int ls_get_status(ls_ctx* c)
{
    if (!c) return LS_EINVAL;
    unsigned st = 0;
    CK(cudaMemcpyAsync(&st, c->d_status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (st & lsk::ST_TIMEOUT) return LS_ETIMEOUT;
    if (st & lsk::ST_NONFINITE) return LS_ENONFINITE;
    if (st) return LS_ECUDA;
    return LS_OK;
}

}  // extern "C"
