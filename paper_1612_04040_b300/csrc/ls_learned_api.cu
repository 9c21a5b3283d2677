// ls_learned_api.cu -- C ABI and host engine of the learned coarse-grid
// corrector (not in the paper): the network's parameters and Adam state,
// the training pairs, one training iteration, and the corrected step used by
// ls_step in LS_LEARNED mode.
//
// Network: 4 convolutions 3x3x3 (3 -> 16 -> 16 -> 16 -> 1 channels), ReLU
// between, BF16 weights and activations on the tensor cores, FP32
// accumulation and FP32 master parameters.  Parameter vector layout: for
// layer l = 0..3: W_l [27][ci_l][co_l] then b_l [co_l].
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "ls_ctx.cuh"

namespace lsk {

namespace {
constexpr int NL = 4;
constexpr int CI[NL] = {3, 16, 16, 16};
constexpr int CO[NL] = {16, 16, 16, 1};

int w_off(int l)
{
    int o = 0;
    for (int k = 0; k < l; ++k) o += 27 * CI[k] * CO[k] + CO[k];
    return o;
}
int b_off(int l) { return w_off(l) + 27 * CI[l] * CO[l]; }
int n_params() { return w_off(NL); }
}  // namespace

struct Pair {
    float* phi = nullptr;   // coarse phi^n, row-major
    float* ref = nullptr;   // reference at n + 1 coarse step (restricted fine run)
    float* F = nullptr;     // coarse speed field
};

struct Learned {
    int nx = 0, ny = 0, nz = 0;
    long long npts = 0;
    float* params = nullptr;
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    int adam_step = 0;
    void* wpack_fwd[NL] = {};
    void* wpack_bwd[NL] = {};
    void* X0 = nullptr;           // features, bf16 [p][16]
    void* A[NL - 1] = {};         // hidden activations
    void* G[NL] = {};             // gradients of the layer outputs (bf16 [p][16])
    float* z = nullptr;           // network output (FP32 [p])
    float* rm_phi = nullptr;      // row-major scratch
    float* rm_phit = nullptr;
    float* rm_F = nullptr;
    int* d_count = nullptr;
    double* d_loss = nullptr;
    unsigned* d_flag = nullptr;
    unsigned long long* d_fallbacks = nullptr;
    CUtensorMap map_X0[2], map_A[NL - 1][2], map_G[NL][2];
    std::vector<Pair> pairs;
    bool initialised = false;
};

void learned_free(Learned* L)
{
    if (!L) return;
    void* ptrs[] = {L->params, L->grads, L->adam_m, L->adam_v, L->X0, L->z, L->rm_phi, L->rm_phit,
                    L->rm_F, L->d_count, L->d_loss, L->d_flag, L->d_fallbacks};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int l = 0; l < NL; ++l) {
        if (L->wpack_fwd[l]) cudaFree(L->wpack_fwd[l]);
        if (L->wpack_bwd[l]) cudaFree(L->wpack_bwd[l]);
        if (L->G[l]) cudaFree(L->G[l]);
        if (l < NL - 1 && L->A[l]) cudaFree(L->A[l]);
    }
    for (auto& p : L->pairs) {
        cudaFree(p.phi);
        cudaFree(p.ref);
        cudaFree(p.F);
    }
    delete L;
}

}  // namespace lsk

using lsk::Learned;

namespace {

#define LCK(expr)                                              \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) return ls_engine_cuda_fail(e_); \
    } while (0)

int ensure_learned(ls_ctx* c, Learned** out)
{
    if (c->batched || c->prec != LS_FP32) return LS_EINVAL;
    const Inst& in = c->in0();
    if (!lsk::conv3_shape_ok(in.nx, in.ny, in.nz)) return LS_EINVAL;
    if (c->learned) {
        *out = c->learned;
        return LS_OK;
    }
    Learned* L = new (std::nothrow) Learned();
    if (!L) return LS_ENOMEM;
    c->learned = L;
    L->nx = in.nx;
    L->ny = in.ny;
    L->nz = in.nz;
    L->npts = (long long)in.nx * in.ny * in.nz;
    const size_t np = (size_t)lsk::n_params();
    const size_t act = (size_t)L->npts * 16 * 2;
    LCK(cudaMalloc(&L->params, np * 4));
    LCK(cudaMalloc(&L->grads, np * 4));
    LCK(cudaMalloc(&L->adam_m, np * 4));
    LCK(cudaMalloc(&L->adam_v, np * 4));
    LCK(cudaMemset(L->adam_m, 0, np * 4));
    LCK(cudaMemset(L->adam_v, 0, np * 4));
    for (int l = 0; l < lsk::NL; ++l) {
        LCK(cudaMalloc(&L->wpack_fwd[l], 27 * 512));
        LCK(cudaMalloc(&L->wpack_bwd[l], 27 * 512));
        LCK(cudaMalloc(&L->G[l], act));
        if (l < lsk::NL - 1) LCK(cudaMalloc(&L->A[l], act));
    }
    LCK(cudaMalloc(&L->X0, act));
    LCK(cudaMemset(L->X0, 0, act));
    LCK(cudaMalloc(&L->z, L->npts * 4));
    LCK(cudaMalloc(&L->rm_phi, L->npts * 4));
    LCK(cudaMalloc(&L->rm_phit, L->npts * 4));
    LCK(cudaMalloc(&L->rm_F, L->npts * 4));
    LCK(cudaMalloc(&L->d_count, sizeof(int)));
    LCK(cudaMalloc(&L->d_loss, sizeof(double)));
    LCK(cudaMalloc(&L->d_flag, sizeof(unsigned)));
    LCK(cudaMalloc(&L->d_fallbacks, sizeof(unsigned long long)));
    LCK(cudaMemset(L->d_flag, 0, sizeof(unsigned)));
    LCK(cudaMemset(L->d_fallbacks, 0, sizeof(unsigned long long)));
    LCK(lsk::make_act_maps(L->map_X0, L->X0, L->nx, L->ny, L->nz));
    for (int l = 0; l < lsk::NL; ++l) {
        LCK(lsk::make_act_maps(L->map_G[l], L->G[l], L->nx, L->ny, L->nz));
        if (l < lsk::NL - 1) LCK(lsk::make_act_maps(L->map_A[l], L->A[l], L->nx, L->ny, L->nz));
    }
    *out = L;
    return LS_OK;
}

int pack_all(ls_ctx* c, Learned* L, bool bwd, cudaStream_t s)
{
    for (int l = 0; l < lsk::NL; ++l) {
        LCK(lsk::launch_pack_weights(L->params + lsk::w_off(l), lsk::CI[l], lsk::CO[l], 0,
                                     L->wpack_fwd[l], s));
        if (bwd)
            LCK(lsk::launch_pack_weights(L->params + lsk::w_off(l), lsk::CI[l], lsk::CO[l], 1,
                                         L->wpack_bwd[l], s));
        c->launches += bwd ? 2 : 1;
    }
    return LS_OK;
}

// forward network on L->X0 -> L->z
int forward(ls_ctx* c, Learned* L, cudaStream_t s)
{
    const CUtensorMap* in = L->map_X0;
    for (int l = 0; l < lsk::NL; ++l) {
        const bool last = l == lsk::NL - 1;
        LCK(lsk::launch_conv3(in, L->wpack_fwd[l], L->params + lsk::b_off(l), nullptr,
                              last ? nullptr : L->A[l], last ? L->z : nullptr, L->nx, L->ny, L->nz,
                              last ? 1 : 0, c->d_status, s));
        ++c->launches;
        if (!last) in = L->map_A[l];
    }
    return LS_OK;
}

}  // namespace

// the corrected step: called right after the plain step wrote phi~ into the
// other buffer (before the swap)
int ls_engine_learned_after_step(ls_ctx* c, cudaStream_t s)
{
    Learned* L = c->learned;
    if (!L || !L->initialised) return LS_ESTATE;
    const Inst& in = c->in0();
    void* src = c->phi[c->cur];
    void* dst = c->phi[c->cur ^ 1];
    LCK(lsk::launch_unpack(src, L->rm_phi, in, 0, s));
    LCK(lsk::launch_unpack(dst, L->rm_phit, in, 0, s));
    const float* F = nullptr;
    if (in.speed_mode == 2) {
        LCK(lsk::launch_unpack(c->F, L->rm_F, in, 0, s));
        F = L->rm_F;
        ++c->launches;
    }
    LCK(lsk::launch_features(L->rm_phi, L->rm_phit, F, (float)in.Fc, (float)in.inv_h, L->npts, L->X0, s));
    c->launches += 3;
    int r = pack_all(c, L, false, s);
    if (r) return r;
    r = forward(c, L, s);
    if (r) return r;
    LCK(lsk::launch_residual((float*)dst, L->z, c->list, c->d_count, in, c->d_sc, (float)in.h,
                             L->d_flag, L->d_fallbacks, s));
    c->launches += 3;
    return LS_OK;
}

extern "C" {

int ls_learned_init(ls_ctx* c, unsigned long long seed)
{
    if (!c) return LS_EINVAL;
    Learned* L = nullptr;
    int r = ensure_learned(c, &L);
    if (r) return r;
    // Kaiming-uniform weights (fan-in 27 ci), zero biases, from a seeded
    // splitmix64 stream on the host
    std::vector<float> p((size_t)lsk::n_params(), 0.f);
    unsigned long long st = seed ^ 0x9e3779b97f4a7c15ull;
    auto next = [&]() {
        unsigned long long z = (st += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int l = 0; l < lsk::NL; ++l) {
        const int n = 27 * lsk::CI[l] * lsk::CO[l];
        double bound = std::sqrt(6.0 / (27.0 * lsk::CI[l]));
        if (l == lsk::NL - 1) bound *= 0.01;  // the corrector starts close to zero
        for (int i = 0; i < n; ++i) p[(size_t)lsk::w_off(l) + i] = (float)((2.0 * next() - 1.0) * bound);
    }
    LCK(cudaMemcpy(L->params, p.data(), p.size() * 4, cudaMemcpyHostToDevice));
    LCK(cudaMemset(L->adam_m, 0, p.size() * 4));
    LCK(cudaMemset(L->adam_v, 0, p.size() * 4));
    L->adam_step = 0;
    L->initialised = true;
    c->graphs.clear();
    return LS_OK;
}

int ls_learned_num_params(long long* n)
{
    if (!n) return LS_EINVAL;
    *n = lsk::n_params();
    return LS_OK;
}

int ls_learned_set_params(ls_ctx* c, const float* src, long long n)
{
    if (!c || !src || n != lsk::n_params()) return LS_EINVAL;
    Learned* L = nullptr;
    int r = ensure_learned(c, &L);
    if (r) return r;
    LCK(cudaMemcpy(L->params, src, (size_t)n * 4, cudaMemcpyHostToDevice));
    L->initialised = true;
    return LS_OK;
}

int ls_learned_get_params(ls_ctx* c, float* dst, long long n)
{
    if (!c || !dst || n != lsk::n_params()) return LS_EINVAL;
    if (!c->learned || !c->learned->initialised) return LS_ESTATE;
    LCK(cudaMemcpy(dst, c->learned->params, (size_t)n * 4, cudaMemcpyDeviceToHost));
    return LS_OK;
}

int ls_learned_add_pair(ls_ctx* c, const float* phi_n, const float* phi_ref, const float* F,
                        int on_device)
{
    if (!c || !phi_n || !phi_ref || !F) return LS_EINVAL;
    Learned* L = nullptr;
    int r = ensure_learned(c, &L);
    if (r) return r;
    lsk::Pair p;
    const size_t bytes = (size_t)L->npts * 4;
    LCK(cudaMalloc(&p.phi, bytes));
    LCK(cudaMalloc(&p.ref, bytes));
    LCK(cudaMalloc(&p.F, bytes));
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    LCK(cudaMemcpyAsync(p.phi, phi_n, bytes, k, c->stream));
    LCK(cudaMemcpyAsync(p.ref, phi_ref, bytes, k, c->stream));
    LCK(cudaMemcpyAsync(p.F, F, bytes, k, c->stream));
    L->pairs.push_back(p);
    return LS_OK;
}

int ls_learned_num_pairs(ls_ctx* c, long long* n)
{
    if (!c || !n) return LS_EINVAL;
    *n = c->learned ? (long long)c->learned->pairs.size() : 0;
    return LS_OK;
}

// one Adam iteration per pair drawn (seeded) from the stored pairs.  The
// plain coarse step uses the fixed dt; the loss is the mean squared error
// of z against (phi_ref - phi~)/h over the points with |phi^n| < gamma,
// gamma = halfwidth * h.
int ls_learned_train(ls_ctx* c, int iters, double lr, double dt, double halfwidth,
                     unsigned long long seed, double* final_loss)
{
    if (!c || iters < 0 || !(lr > 0) || !(dt > 0) || !(halfwidth > 0)) return LS_EINVAL;
    Learned* L = c->learned;
    if (!L || !L->initialised || L->pairs.empty()) return LS_ESTATE;
    cudaStream_t s = c->stream;
    const Inst in = c->in0();
    const float inv_h = (float)in.inv_h;
    const float gamma = (float)(halfwidth * in.h);
    unsigned long long st = seed;
    double loss = 0.0;
    // the context's phi / speed are used as scratch for the plain coarse
    // step; they are marked stale afterwards
    const bool fd = c->full_domain;
    c->full_domain = true;
    for (int it = 0; it < iters; ++it) {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        const lsk::Pair& P = L->pairs[(size_t)((st >> 33) % L->pairs.size())];
        // phi~ = plain step of phi^n with the pair's speed
        int r = ls_engine_pack(c, in, P.phi, 1, c->phi[0]);
        if (r) return r;
        LCK(cudaMemcpyAsync(c->phi[1], c->phi[0], (size_t)L->npts * 4, cudaMemcpyDeviceToDevice, s));
        c->cur = 0;
        c->inst_phi_set[0] = 1;
        r = ls_set_speed(c, P.F, 1);
        if (r) return r;
        const int mode = c->step_mode;
        c->step_mode = LS_PLAIN;
        r = ls_step(c, 1, dt, LS_DT_FIXED, 0, nullptr);
        c->step_mode = mode;
        if (r) return r;
        LCK(lsk::launch_unpack(c->phi[c->cur], L->rm_phit, in, 0, s));
        LCK(lsk::launch_features(P.phi, L->rm_phit, P.F, 0.f, inv_h, L->npts, L->X0, s));
        r = pack_all(c, L, true, s);
        if (r) return r;
        r = forward(c, L, s);
        if (r) return r;
        LCK(cudaMemsetAsync(L->d_count, 0, sizeof(int), s));
        LCK(cudaMemsetAsync(L->d_loss, 0, sizeof(double), s));
        LCK(lsk::launch_count_mask(P.phi, gamma, L->npts, L->d_count, s));
        LCK(lsk::launch_loss_grad(L->z, P.phi, L->rm_phit, P.ref, inv_h, gamma, L->d_count, L->npts,
                                  L->G[lsk::NL - 1], L->d_loss, s));
        LCK(cudaMemsetAsync(L->grads, 0, (size_t)lsk::n_params() * 4, s));
        for (int l = lsk::NL - 1; l >= 0; --l) {
            const void* xin = (l == 0) ? L->X0 : L->A[l - 1];
            LCK(lsk::launch_conv3_wgrad(xin, L->G[l], L->nx, L->ny, L->nz, lsk::CI[l], lsk::CO[l],
                                        L->grads + lsk::w_off(l), L->grads + lsk::b_off(l), s));
            if (l > 0)
                LCK(lsk::launch_conv3(L->map_G[l], L->wpack_bwd[l], nullptr, L->A[l - 1],
                                      L->G[l - 1], nullptr, L->nx, L->ny, L->nz, 2, c->d_status, s));
        }
        LCK(lsk::launch_adam(L->params, L->grads, L->adam_m, L->adam_v, lsk::n_params(), (float)lr,
                             ++L->adam_step, s));
        if (it == iters - 1 && final_loss) {
            LCK(cudaMemcpyAsync(&loss, L->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
            LCK(cudaStreamSynchronize(s));
            *final_loss = loss;
        }
    }
    c->full_domain = fd;
    c->band_valid = false;
    c->core_fresh = false;
    c->inst_phi_set[0] = 0;  // phi holds a training sample now
    c->graphs.clear();
    return LS_OK;
}

int ls_set_step_mode(ls_ctx* c, int mode)
{
    if (!c || (mode != LS_PLAIN && mode != LS_LEARNED)) return LS_EINVAL;
    if (mode == LS_LEARNED && (!c->learned || !c->learned->initialised)) return LS_ESTATE;
    if (mode == LS_LEARNED && c->scheme != LS_SCHEME_PLAIN) return LS_ESTATE;
    c->step_mode = mode;
    return LS_OK;
}

int ls_learned_fallbacks(ls_ctx* c, unsigned long long* n)
{
    if (!c || !n) return LS_EINVAL;
    *n = 0;
    if (!c->learned) return LS_OK;
    LCK(cudaMemcpyAsync(n, c->learned->d_fallbacks, sizeof(*n), cudaMemcpyDeviceToHost, c->stream));
    LCK(cudaStreamSynchronize(c->stream));
    return LS_OK;
}

// ---- layer primitives on caller buffers (tests, custom pipelines) -------

int ls_conv3_bf16(const void* x, int nx, int ny, int nz, const float* W, int ci, int co,
                  const float* bias, int mode, const void* mask, void* out, void* work,
                  unsigned* status, void* stream)
{
    if (!x || !W || !out || !work || !status) return LS_EINVAL;
    if (ci < 1 || ci > 16 || co < 1 || co > 16 || mode < 0 || mode > 2) return LS_EINVAL;
    if (!lsk::conv3_shape_ok(nx, ny, nz)) return LS_EINVAL;
    if (mode != 2 && !bias) return LS_EINVAL;
    if (mode == 2 && !mask) return LS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    CUtensorMap maps[2];
    LCK(lsk::make_act_maps(maps, x, nx, ny, nz));
    LCK(lsk::launch_pack_weights(W, ci, co, mode == 2 ? 1 : 0, work, s));
    LCK(lsk::launch_conv3(maps, work, bias, mask, mode == 1 ? nullptr : out,
                          mode == 1 ? (float*)out : nullptr, nx, ny, nz, mode, status, s));
    return LS_OK;
}

int ls_conv3_wgrad(const void* x, const void* dy, int nx, int ny, int nz, int ci, int co,
                   float* dW, float* db, void* stream)
{
    if (!x || !dy || !dW || ci < 1 || ci > 16 || co < 1 || co > 16) return LS_EINVAL;
    if (nx % 64 || ny < 1 || nz < 1) return LS_EINVAL;
    LCK(lsk::launch_conv3_wgrad(x, dy, nx, ny, nz, ci, co, dW, db, (cudaStream_t)stream));
    return LS_OK;
}

int ls_restrict4(const float* fine, int nfx, int nfy, int nfz, float* coarse, void* stream)
{
    if (!fine || !coarse || nfx < 4 || nfy < 4 || nfz < 4 || nfx % 4 || nfy % 4 || nfz % 4)
        return LS_EINVAL;
    LCK(lsk::launch_restrict4(fine, nfx, nfy, nfz, coarse, (cudaStream_t)stream));
    return LS_OK;
}

}  // extern "C"
