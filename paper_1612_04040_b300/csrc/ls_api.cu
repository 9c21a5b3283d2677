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
//   2. rebuild = dilation (+ copy of tiles leaving the active set into the
//      other ping-pong buffer) -> scan of block counts -> ascending scatter of
//      active ids, folding max|F| of the active tiles -> dt in FP64;
//   3. one launch of the stencil over the active list, src -> dst, swap.
// Nothing is read back to the host inside ls_step: counts, M and dt stay in
// device memory and the persistent stencil grid reads the count there.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ls.h"
#include "ls_internal.cuh"

using lsk::Inst;

static thread_local int g_last_cuda_error = 0;

struct ls_ctx {
    int prec = 0;
    size_t esize = 4;
    Inst in{};                    // single instance (n_inst == 1)
    long long ntiles = 0;
    size_t npts = 0;
    cudaStream_t stream = nullptr;
    void* phi[2] = {nullptr, nullptr};
    int cur = 0;
    void* F = nullptr;            // bricked speed field (lazy)
    void* tile_maxF = nullptr;    // per-tile max |F| (lazy)
    void* staging = nullptr;      // row-major staging buffer (lazy)
    uint8_t* core = nullptr;
    uint8_t* act = nullptr;
    int* list = nullptr;
    uint8_t* list_info = nullptr;
    uint8_t* tile_sgn = nullptr;  // per-tile sign code of a speed field (lazy)
    int* d_count = nullptr;
    int* block_counts = nullptr;
    int nblocks = 0;
    lsk::StepScalars* d_sc = nullptr;
    unsigned long long* d_Mbits = nullptr;
    unsigned long long* d_updates = nullptr;
    unsigned* d_status = nullptr;
    unsigned* d_nonfinite = nullptr;
    // host-side state
    bool phi_set = false;
    bool band_valid = false;
    bool core_fresh = false;
    bool full_domain = false;
    bool have_halfwidth = false;
    double halfwidth = 0.0;
    int since_rebuild = 0;
    int dt_mode = LS_DT_FIXED;
    double dt_value = 0.0;
    // profiling
    unsigned long long launches = 0;
    unsigned long long stencil_launches = 0;
    bool profiling = false;
    double stencil_ms = 0.0;
    unsigned long long stencil_timed = 0;
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
};

namespace {

int cuda_fail(cudaError_t e)
{
    g_last_cuda_error = (int)e;
    if (e == cudaErrorMemoryAllocation) return LS_ENOMEM;
    return LS_ECUDA;
}

#define CK(expr)                                    \
    do {                                            \
        cudaError_t e_ = (expr);                    \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

// a library kernel launch: counted, then checked
#define KL(c, expr)          \
    do {                     \
        ++(c)->launches;     \
        CK(expr);            \
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
        CK(cudaEventElapsedTime(&ms, p.first, p.second));
        c->stencil_ms += ms;
        c->stencil_timed += 1;
        c->ev_free.push_back(p.first);
        c->ev_free.push_back(p.second);
    }
    c->ev_pending.clear();
    return LS_OK;
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
    for (auto& p : c->ev_pending) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    for (auto e : c->ev_free) cudaEventDestroy(e);
    void* ptrs[] = {c->phi[0], c->phi[1], c->F, c->tile_maxF, c->staging, c->core, c->act,
                    c->list, c->list_info, c->tile_sgn, c->d_count, c->block_counts, c->d_sc, c->d_Mbits, c->d_updates,
                    c->d_status, c->d_nonfinite};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

size_t grid_bytes(const ls_ctx* c) { return c->npts * c->esize; }

int ensure_staging(ls_ctx* c)
{
    if (!c->staging) CK(dalloc(&c->staging, grid_bytes(c)));
    return LS_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// pack a row-major source (host or device) into the bricked buffer dst;
// returns LS_ENONFINITE if any value is NaN/Inf (after a stream sync)
int pack_from(ls_ctx* c, const void* src, int on_device, void* dst)
{
    const void* dsrc = src;
    if (!on_device) {
        int r = ensure_staging(c);
        if (r) return r;
        CK(cudaMemcpyAsync(c->staging, src, grid_bytes(c), cudaMemcpyHostToDevice, c->stream));
        dsrc = c->staging;
    } else if (!aligned16(src)) {
        return LS_EINVAL;
    }
    CK(cudaMemsetAsync(c->d_nonfinite, 0, sizeof(unsigned), c->stream));
    KL(c, lsk::launch_pack(dsrc, dst, c->in, c->prec, c->d_nonfinite, c->stream));
    unsigned bad = 0;
    CK(cudaMemcpyAsync(&bad, c->d_nonfinite, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return bad ? LS_ENONFINITE : LS_OK;
}

unsigned const_sign_bits(const ls_ctx* c)
{
    return c->in.Fc >= 0.0 ? lsk::SG_POS : lsk::SG_NEG;
}

const uint8_t* sign_table(const ls_ctx* c)
{
    return c->in.speed_mode == 2 ? c->tile_sgn : nullptr;
}

int rebuild(ls_ctx* c, bool full_scan)
{
    cudaStream_t s = c->stream;
    void* cur = c->phi[c->cur];
    void* other = c->phi[c->cur ^ 1];
    if (full_scan || !c->core_fresh)
        KL(c, lsk::launch_classify_all(cur, c->core, nullptr, nullptr, c->in, c->ntiles, c->prec, s));
    KL(c, lsk::launch_dilate(c->core, c->act, c->block_counts, nullptr, nullptr, c->in, c->ntiles,
                             s));
    KL(c, lsk::launch_scan(c->block_counts, c->nblocks, c->d_count, s));
    const void* tmf = (c->in.speed_mode == 2) ? c->tile_maxF : nullptr;
    KL(c, lsk::launch_scatter(c->act, c->block_counts, c->list, c->list_info, sign_table(c),
                              const_sign_bits(c), c->in, c->ntiles, tmf, c->prec, c->d_Mbits, cur,
                              other, s));
    KL(c, lsk::launch_set_dt(c->d_sc, 1, nullptr, c->in, c->dt_mode, c->dt_value, 1, c->prec,
                          c->d_Mbits, c->d_count, 0, s));
    c->band_valid = true;
    c->core_fresh = false;
    c->since_rebuild = 0;
    return LS_OK;
}

int full_domain_bound(ls_ctx* c)
{
    // every tile counts as active, so a later switch back to a band copies
    // every tile that leaves the active set into the other buffer
    CK(cudaMemsetAsync(c->act, 1, c->ntiles, c->stream));
    KL(c, lsk::launch_full_list(c->list, c->list_info, sign_table(c), const_sign_bits(c), c->in,
                                c->ntiles, c->d_count, c->stream));
    if (c->in.speed_mode == 2)
        KL(c, lsk::launch_max_all(c->tile_maxF, c->ntiles, c->prec, c->d_Mbits, c->stream));
    KL(c, lsk::launch_set_dt(c->d_sc, 1, nullptr, c->in, c->dt_mode, c->dt_value, 1, c->prec,
                          c->d_Mbits, nullptr, c->ntiles, c->stream));
    c->band_valid = true;
    return LS_OK;
}

}  // namespace

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
    default: return "unknown status";
    }
}

int ls_last_cuda_error(void) { return g_last_cuda_error; }

int ls_create(int nx, int ny, int nz, double h, int precision, ls_ctx** out)
{
    if (!out) return LS_EINVAL;
    *out = nullptr;
    if (nx < 8 || ny < 8 || nz < 8 || nx % 8 || ny % 8 || nz % 8) return LS_EINVAL;
    if ((long long)nx * ny * nz > (1ll << 31)) return LS_EINVAL;
    if (!(h > 0.0) || !std::isfinite(h)) return LS_EINVAL;
    if (precision != LS_FP32 && precision != LS_FP64) return LS_EINVAL;
    ls_ctx* c = new (std::nothrow) ls_ctx();
    if (!c) return LS_ENOMEM;
    c->prec = precision;
    c->esize = precision == LS_FP32 ? 4 : 8;
    Inst& in = c->in;
    in.nx = nx; in.ny = ny; in.nz = nz;
    in.tnx = nx / 8; in.tny = ny / 8; in.tnz = nz / 8;
    in.tile_base = 0;
    in.ntiles = (long long)in.tnx * in.tny * in.tnz;
    in.h = h;
    in.inv_h = 1.0 / h;
    in.gamma = 0.0;
    in.Fc = 0.0;
    in.speed_mode = 0;
    in.pow2h = is_pow2(h) ? 1 : 0;
    in.bc = LS_BC_EXTRAPOLATE;
    c->ntiles = in.ntiles;
    c->npts = (size_t)nx * ny * nz;
    c->nblocks = (int)((c->ntiles + 255) / 256);
    if (c->nblocks > 1024 * 32) { delete c; return LS_EINVAL; }
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess && r != cudaSuccess) e = r; };
    A(dalloc(&c->phi[0], grid_bytes(c)));
    A(dalloc(&c->phi[1], grid_bytes(c)));
    A(dalloc(&c->core, c->ntiles));
    A(dalloc(&c->act, c->ntiles));
    A(dalloc(&c->list, c->ntiles * sizeof(int)));
    A(dalloc(&c->list_info, c->ntiles));
    A(dalloc(&c->d_count, sizeof(int)));
    A(dalloc(&c->block_counts, c->nblocks * sizeof(int)));
    A(dalloc(&c->d_sc, sizeof(lsk::StepScalars)));
    A(dalloc(&c->d_Mbits, sizeof(unsigned long long)));
    A(dalloc(&c->d_updates, sizeof(unsigned long long)));
    A(dalloc(&c->d_status, sizeof(unsigned)));
    A(dalloc(&c->d_nonfinite, sizeof(unsigned)));
    if (e == cudaSuccess) {
        A(cudaMemset(c->core, 0, c->ntiles));
        A(cudaMemset(c->act, 0, c->ntiles));
        A(cudaMemset(c->d_count, 0, sizeof(int)));
        A(cudaMemset(c->d_sc, 0, sizeof(lsk::StepScalars)));
        A(cudaMemset(c->d_Mbits, 0, sizeof(unsigned long long)));
        A(cudaMemset(c->d_updates, 0, sizeof(unsigned long long)));
        A(cudaMemset(c->d_status, 0, sizeof(unsigned)));
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
    return LS_OK;
}

int ls_set_bc(ls_ctx* c, int bc)
{
    if (!c || (bc != LS_BC_EXTRAPOLATE && bc != LS_BC_NEUMANN)) return LS_EINVAL;
    c->in.bc = bc;
    return LS_OK;
}

int ls_set_phi(ls_ctx* c, const void* src, int on_device)
{
    if (!c || !src) return LS_EINVAL;
    c->band_valid = false;
    c->core_fresh = false;
    int r = pack_from(c, src, on_device, c->phi[0]);
    if (r) { c->phi_set = false; return r; }
    CK(cudaMemcpyAsync(c->phi[1], c->phi[0], grid_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
    c->cur = 0;
    c->phi_set = true;
    return LS_OK;
}

int ls_set_speed(ls_ctx* c, const void* src, int on_device)
{
    if (!c || !src) return LS_EINVAL;
    if (!c->F) CK(dalloc(&c->F, grid_bytes(c)));
    if (!c->tile_maxF) CK(dalloc(&c->tile_maxF, c->ntiles * c->esize));
    if (!c->tile_sgn) CK(dalloc(&c->tile_sgn, c->ntiles));
    c->band_valid = false;
    c->core_fresh = false;
    int r = pack_from(c, src, on_device, c->F);
    if (r) { c->in.speed_mode = 0; return r; }
    KL(c, lsk::launch_tile_speed(c->F, c->tile_maxF, c->tile_sgn, c->ntiles, c->prec, c->stream));
    c->in.speed_mode = 2;
    return LS_OK;
}

int ls_set_speed_const(ls_ctx* c, double F)
{
    if (!c) return LS_EINVAL;
    if (!std::isfinite(F)) return LS_ENONFINITE;
    c->in.Fc = F;
    c->in.speed_mode = 1;
    c->band_valid = false;
    c->core_fresh = false;
    return LS_OK;
}

int ls_set_full_domain(ls_ctx* c, int on)
{
    if (!c) return LS_EINVAL;
    c->full_domain = on != 0;
    c->band_valid = false;
    c->core_fresh = false;
    return LS_OK;
}

int ls_band_rebuild(ls_ctx* c, double halfwidth, long long* n_active)
{
    if (!c) return LS_EINVAL;
    if (!(halfwidth > 0.0) || !std::isfinite(halfwidth)) return LS_EINVAL;
    if (!c->phi_set) return LS_ESTATE;
    c->halfwidth = halfwidth;
    c->have_halfwidth = true;
    c->in.gamma = halfwidth * c->in.h;
    int r = rebuild(c, true);
    if (r) return r;
    if (n_active) {
        int n = 0;
        CK(cudaMemcpyAsync(&n, c->d_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        *n_active = n;
    }
    return LS_OK;
}

int ls_step(ls_ctx* c, int nsteps, double value, int dt_mode, int rebuild_every, double* last_dt)
{
    if (!c) return LS_EINVAL;
    if (nsteps < 0 || rebuild_every < 0) return LS_EINVAL;
    if (dt_mode != LS_DT_FIXED && dt_mode != LS_DT_CFL) return LS_EINVAL;
    if (!(value > 0.0) || !std::isfinite(value)) return LS_EINVAL;
    if (!c->phi_set || c->in.speed_mode == 0) return LS_ESTATE;
    if (!c->full_domain && !c->have_halfwidth) return LS_ESTATE;
    cudaStream_t s = c->stream;
    c->dt_mode = dt_mode;
    c->dt_value = value;
    bool dt_pending = true;
    for (int k = 0; k < nsteps; ++k) {
        bool rebuilt = false;
        if (c->full_domain) {
            if (!c->band_valid) {
                int r = full_domain_bound(c);
                if (r) return r;
                rebuilt = true;
            }
        } else if (!c->band_valid) {
            int r = rebuild(c, true);
            if (r) return r;
            rebuilt = true;
        } else if (rebuild_every > 0 && c->since_rebuild >= rebuild_every) {
            int r = rebuild(c, false);
            if (r) return r;
            rebuilt = true;
        }
        if (dt_pending && !rebuilt)
            KL(c, lsk::launch_set_dt(c->d_sc, 1, nullptr, c->in, dt_mode, value, 0, c->prec,
                                  c->d_Mbits, nullptr, 0, s));
        dt_pending = false;
        const bool classify = !c->full_domain && rebuild_every > 0 &&
                              c->since_rebuild + 1 >= rebuild_every;
        lsk::StepArgs a{};
        a.src = c->phi[c->cur];
        a.dst = c->phi[c->cur ^ 1];
        a.F = (c->in.speed_mode == 2) ? c->F : nullptr;
        a.list = c->list;
        a.info = c->list_info;
        a.count = c->d_count;
        a.sc = c->d_sc;
        a.core = classify ? c->core : nullptr;
        a.updates = c->d_updates;
        a.in = c->in;
        int grid = lsk::step_grid_size(c->prec, classify);
        if (c->full_domain && grid > c->ntiles) grid = (int)c->ntiles;
        if (c->profiling && c->ev_pending.size() >= 4096) {
            int r = drain_events(c);
            if (r) return r;
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (c->profiling) {
            CK(take_event(c, &e0));
            CK(take_event(c, &e1));
            CK(cudaEventRecord(e0, s));
        }
        KL(c, lsk::launch_step(a, c->prec, grid, s));
        ++c->stencil_launches;
        if (c->profiling) {
            CK(cudaEventRecord(e1, s));
            c->ev_pending.emplace_back(e0, e1);
        }
        c->cur ^= 1;
        c->since_rebuild += 1;
        c->core_fresh = classify;
    }
    if (last_dt) {
        lsk::StepScalars sc;
        CK(cudaMemcpyAsync(&sc, c->d_sc, sizeof(sc), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        *last_dt = sc.dt;
    }
    return LS_OK;
}

int ls_get_phi(ls_ctx* c, void* dst, int on_device)
{
    if (!c || !dst) return LS_EINVAL;
    if (!c->phi_set) return LS_ESTATE;
    if (on_device) {
        if (!aligned16(dst)) return LS_EINVAL;
        KL(c, lsk::launch_unpack(c->phi[c->cur], dst, c->in, c->prec, c->stream));
    } else {
        int r = ensure_staging(c);
        if (r) return r;
        KL(c, lsk::launch_unpack(c->phi[c->cur], c->staging, c->in, c->prec, c->stream));
        CK(cudaMemcpyAsync(dst, c->staging, grid_bytes(c), cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return LS_OK;
}

int ls_get_active_tiles(ls_ctx* c, int* dst, long long cap, long long* n)
{
    if (!c || !n || cap < 0 || (cap > 0 && !dst)) return LS_EINVAL;
    if (!c->band_valid && !c->full_domain) return LS_ESTATE;
    if (c->full_domain) {
        *n = c->ntiles;
        long long k = cap < c->ntiles ? cap : c->ntiles;
        for (long long i = 0; i < k; ++i) dst[i] = (int)i;
        return LS_OK;
    }
    int cnt = 0;
    CK(cudaMemcpyAsync(&cnt, c->d_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *n = cnt;
    long long k = cap < cnt ? cap : cnt;
    if (k > 0) {
        CK(cudaMemcpyAsync(dst, c->list, k * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
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
    c->profiling = on != 0;
    return LS_OK;
}

int ls_get_profile(ls_ctx* c, ls_profile* out)
{
    if (!c || !out) return LS_EINVAL;
    int r = drain_events(c);
    if (r) return r;
    out->kernel_launches = c->launches;
    out->stencil_launches = c->stencil_launches;
    out->stencil_ms = c->stencil_ms;
    out->stencil_timed = c->stencil_timed;
    return LS_OK;
}

int ls_reset_profile(ls_ctx* c)
{
    if (!c) return LS_EINVAL;
    int r = drain_events(c);
    if (r) return r;
    c->launches = 0;
    c->stencil_launches = 0;
    c->stencil_ms = 0.0;
    c->stencil_timed = 0;
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
