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
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
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
    int* d_blist = nullptr;       // convolution blocks near the band (corrected step)
    int* d_bcount = nullptr;
    CUtensorMap map_X0[2], map_A[NL - 1][2], map_G[NL][2];
    std::vector<Pair> pairs;
    bool initialised = false;
    bool fwd_packed = false;      // wpack_fwd holds the current parameters
};

void learned_free(Learned* L)
{
    if (!L) return;
    void* ptrs[] = {L->params, L->grads, L->adam_m, L->adam_v, L->X0, L->z, L->rm_phi, L->rm_phit,
                    L->rm_F, L->d_count, L->d_loss, L->d_flag, L->d_fallbacks, L->d_blist,
                    L->d_bcount};
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
    // activations start at zero: a step that computes the network only near
    // the band reads finite values everywhere
    for (int l = 0; l < lsk::NL; ++l) {
        LCK(cudaMalloc(&L->wpack_fwd[l], 27 * 512));
        LCK(cudaMalloc(&L->wpack_bwd[l], 27 * 512));
        LCK(cudaMalloc(&L->G[l], act));
        LCK(cudaMemset(L->G[l], 0, act));
        if (l < lsk::NL - 1) {
            LCK(cudaMalloc(&L->A[l], act));
            LCK(cudaMemset(L->A[l], 0, act));
        }
    }
    LCK(cudaMalloc(&L->X0, act));
    LCK(cudaMemset(L->X0, 0, act));
    LCK(cudaMalloc(&L->z, L->npts * 4));
    LCK(cudaMemset(L->z, 0, L->npts * 4));
    LCK(cudaMalloc(&L->d_blist, sizeof(int) * (size_t)lsk::conv3_blocks(L->nx, L->ny, L->nz)));
    LCK(cudaMalloc(&L->d_bcount, sizeof(int)));
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
    // inference packs once per parameter change; training every iteration
    if (!bwd && L->fwd_packed) return LS_OK;
    L->fwd_packed = !bwd;
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

// forward network on L->X0 -> L->z, on every block or on the listed ones
int forward(ls_ctx* c, Learned* L, cudaStream_t s, bool band_only = false)
{
    const CUtensorMap* in = L->map_X0;
    for (int l = 0; l < lsk::NL; ++l) {
        const bool last = l == lsk::NL - 1;
        LCK(lsk::launch_conv3(in, L->wpack_fwd[l], L->params + lsk::b_off(l), nullptr,
                              last ? nullptr : L->A[l], last ? L->z : nullptr, L->nx, L->ny, L->nz,
                              last ? 1 : 0, c->d_status, s, band_only ? L->d_blist : nullptr,
                              band_only ? L->d_bcount : nullptr));
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
    // features straight from the bricked phi^n, phi~ and F
    LCK(lsk::launch_features_bricked((const float*)src, (const float*)dst,
                                     in.speed_mode == 2 ? (const float*)c->F : nullptr, in, L->X0, s));
    c->launches += 1;
    int r = pack_all(c, L, false, s);
    if (r) return r;
    LCK(lsk::launch_block_list(c->act, in, L->d_blist, L->d_bcount, s));
    c->launches += 1;
    r = forward(c, L, s, true);
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
    L->fwd_packed = false;
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
    L->fwd_packed = false;
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
int ls_learned_train_stored(ls_ctx* c, int iters, double lr, double dt, double halfwidth,
                            unsigned long long seed, double* final_loss)
{
    if (!c || iters < 0 || !(lr > 0) || !(dt > 0) || !(halfwidth > 0)) return LS_EINVAL;
    Learned* L = c->learned;
    if (!L || !L->initialised || L->pairs.empty()) return LS_ESTATE;
    cudaStream_t s = c->stream;
    const Inst in = c->in0();
    const float inv_h = (float)in.inv_h;
    const double gamma = halfwidth * in.h;
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
                                        L->grads + lsk::w_off(l), L->grads + lsk::b_off(l),
                                        c->d_status, s));
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
    L->fwd_packed = false;
    c->band_valid = false;
    c->core_fresh = false;
    c->inst_phi_set[0] = 0;  // phi holds a training sample now
    c->graphs.clear();
    return LS_OK;
}

int ls_learned_load(ls_ctx* c, const void* bf16_weights, size_t bytes)
{
    if (!c || !bf16_weights || bytes != (size_t)lsk::n_params() * 2) return LS_EINVAL;
    Learned* L = nullptr;
    int r = ensure_learned(c, &L);
    if (r) return r;
    const uint16_t* w = (const uint16_t*)bf16_weights;
    std::vector<float> p((size_t)lsk::n_params());
    for (size_t i = 0; i < p.size(); ++i) {
        const uint32_t u = (uint32_t)w[i] << 16;  // a BF16 value is the top half of an FP32
        std::memcpy(&p[i], &u, 4);
    }
    LCK(cudaMemcpy(L->params, p.data(), p.size() * 4, cudaMemcpyHostToDevice));
    LCK(cudaMemset(L->adam_m, 0, p.size() * 4));
    LCK(cudaMemset(L->adam_v, 0, p.size() * 4));
    L->adam_step = 0;
    L->initialised = true;
    L->fwd_packed = false;
    c->graphs.clear();
    return LS_OK;
}

int ls_learned_save(ls_ctx* c, void* bf16_weights, size_t bytes)
{
    if (!c || !bf16_weights || bytes != (size_t)lsk::n_params() * 2) return LS_EINVAL;
    if (!c->learned || !c->learned->initialised) return LS_ESTATE;
    std::vector<float> p((size_t)lsk::n_params());
    LCK(cudaMemcpy(p.data(), c->learned->params, p.size() * 4, cudaMemcpyDeviceToHost));
    uint16_t* w = (uint16_t*)bf16_weights;
    for (size_t i = 0; i < p.size(); ++i) {
        uint32_t u;
        std::memcpy(&u, &p[i], 4);
        if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) {
            w[i] = (uint16_t)((u >> 16) | 0x40u);  // NaN stays NaN
        } else {
            u += 0x7fffu + ((u >> 16) & 1u);       // round to nearest, ties to even
            w[i] = (uint16_t)(u >> 16);
        }
    }
    return LS_OK;
}

int ls_learned_get_pair(ls_ctx* c, long long i, float* phi_n, float* phi_ref, float* F, int on_device)
{
    if (!c || !phi_n || !phi_ref || !F) return LS_EINVAL;
    if (!c->learned || i < 0 || i >= (long long)c->learned->pairs.size()) return LS_EINVAL;
    const lsk::Pair& P = c->learned->pairs[(size_t)i];
    const size_t bytes = (size_t)c->learned->npts * 4;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    LCK(cudaMemcpyAsync(phi_n, P.phi, bytes, k, c->stream));
    LCK(cudaMemcpyAsync(phi_ref, P.ref, bytes, k, c->stream));
    LCK(cudaMemcpyAsync(F, P.F, bytes, k, c->stream));
    LCK(cudaStreamSynchronize(c->stream));
    return LS_OK;
}

}  // extern "C"

namespace {

// "key=value" items separated by ',' or ';'
struct Spec {
    double dt = -1.0, halfwidth = 6.0, cfl = 0.5;
    unsigned long long seed = 0, gen_seed = 1;
    int fine = 0, problems = 8, pairs = 24;
};

int parse_spec(const char* text, Spec* sp)
{
    if (!text) return LS_OK;
    std::string t(text);
    size_t pos = 0;
    while (pos <= t.size()) {
        size_t end = t.find_first_of(",;", pos);
        if (end == std::string::npos) end = t.size();
        std::string item = t.substr(pos, end - pos);
        pos = end + 1;
        const size_t a = item.find_first_not_of(" \t");
        if (a == std::string::npos) continue;
        item = item.substr(a, item.find_last_not_of(" \t") - a + 1);
        const size_t eq = item.find('=');
        if (eq == std::string::npos) return LS_EINVAL;
        std::string key = item.substr(0, eq), val = item.substr(eq + 1);
        while (!key.empty() && (key.back() == ' ' || key.back() == '\t')) key.pop_back();
        while (!val.empty() && (val.front() == ' ' || val.front() == '\t')) val.erase(0, 1);
        if (val.empty()) return LS_EINVAL;
        char* e = nullptr;
        if (key == "source") {
            if (val == "stored") sp->fine = 0;
            else if (val == "fine") sp->fine = 1;
            else return LS_EINVAL;
            continue;
        }
        if (key == "seed" || key == "gen_seed") {
            const unsigned long long v = std::strtoull(val.c_str(), &e, 10);
            if (*e) return LS_EINVAL;
            (key == "seed" ? sp->seed : sp->gen_seed) = v;
            continue;
        }
        if (key == "problems" || key == "pairs") {
            const long v = std::strtol(val.c_str(), &e, 10);
            if (*e || v < 1 || v > 100000) return LS_EINVAL;
            (key == "problems" ? sp->problems : sp->pairs) = (int)v;
            continue;
        }
        const double v = std::strtod(val.c_str(), &e);
        if (*e || !std::isfinite(v) || !(v > 0.0)) return LS_EINVAL;
        if (key == "dt") sp->dt = v;
        else if (key == "halfwidth") sp->halfwidth = v;
        else if (key == "cfl") sp->cfl = v;
        else return LS_EINVAL;
    }
    return LS_OK;
}

// seeded splitmix64 stream (uniform doubles in [0, 1))
struct Rng {
    unsigned long long st;
    explicit Rng(unsigned long long s) : st(s ^ 0x6a09e667f3bcc909ull) {}
    double next()
    {
        unsigned long long z = (st += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    }
    double uniform(double a, double b) { return a + (b - a) * next(); }
};

#define GCK(expr)                                                     \
    do {                                                              \
        int r_ = (expr);                                              \
        if (r_ != LS_OK) { ls_destroy(fine); cudaFree(scratch); return r_; } \
    } while (0)

// Training pairs from plain runs on the 4x finer grid, restricted to this
// context's grid: per problem a seeded sphere union (2..5 spheres inside the
// middle 60 % of the box) and an 8-mode Fourier speed with |k|_inf <= 2 and
// |F| <= 1; the fine band is 4x as wide in fine cells; dt_f = cfl * h_f and
// every 4 fine steps give one pair (R(phi_f^n), R(phi_f^{n+4}), R(F_f)).
int generate_pairs(ls_ctx* c, Learned* L, const Spec& sp)
{
    const Inst in = c->in0();
    const int fx = 4 * in.nx, fy = 4 * in.ny, fz = 4 * in.nz;
    const double hf = in.h / 4.0;
    const double box[3] = {fx * hf, fy * hf, fz * hf};
    const double bmin = std::fmin(box[0], std::fmin(box[1], box[2]));
    ls_ctx* fine = nullptr;
    float* scratch = nullptr;
    int r = ls_create(fx, fy, fz, hf, LS_FP32, &fine);
    if (r) return r;
    const size_t fpts = (size_t)fx * fy * fz;
    if (cudaMalloc(&scratch, fpts * 4) != cudaSuccess) {
        ls_destroy(fine);
        return LS_ENOMEM;
    }
    GCK(ls_set_stream(fine, c->stream));
    const size_t cbytes = (size_t)L->npts * 4;
    Rng g(sp.gen_seed);
    for (int prob = 0; prob < sp.problems; ++prob) {
        const int k = 2 + (int)(g.next() * 4.0);
        std::vector<double> sph(1 + 4 * (size_t)k);
        sph[0] = k;
        const double rmax = 0.35 * bmin;
        for (int i = 0; i < k; ++i) {
            for (int d = 0; d < 3; ++d) sph[1 + 4 * i + d] = g.uniform(0.2 * box[d], 0.8 * box[d]);
            sph[1 + 4 * i + 3] = g.uniform(0.3 * rmax, rmax);
        }
        std::vector<double> four(1 + 5 * 8);
        four[0] = 8;
        for (int m = 0; m < 8;) {
            int kv[3];
            for (int d = 0; d < 3; ++d) kv[d] = (int)(g.next() * 5.0) - 2;
            if (!kv[0] && !kv[1] && !kv[2]) continue;
            double* q = &four[1 + 5 * m];
            q[0] = g.uniform(-1.0, 1.0);
            q[1] = kv[0];
            q[2] = kv[1];
            q[3] = kv[2];
            q[4] = g.uniform(0.0, 6.283185307179586);
            ++m;
        }
        GCK(ls_init_phi(fine, LS_SHAPE_SPHERES, sph.data(), (int)sph.size()));
        GCK(ls_init_speed(fine, LS_SPEED_FOURIER, four.data(), (int)four.size()));
        GCK(ls_band_rebuild(fine, 4.0 * sp.halfwidth, nullptr));
        cudaStream_t s = c->stream;
        // coarse speed and the first state
        lsk::Pair P;
        auto alloc_pair = [&](lsk::Pair& q) -> int {
            if (cudaMalloc(&q.phi, cbytes) != cudaSuccess || cudaMalloc(&q.ref, cbytes) != cudaSuccess ||
                cudaMalloc(&q.F, cbytes) != cudaSuccess) {
                cudaFree(q.phi); cudaFree(q.ref); cudaFree(q.F);
                return LS_ENOMEM;
            }
            return LS_OK;
        };
        float* Fc = nullptr;
        float* prev = nullptr;
        if (cudaMalloc(&Fc, cbytes) != cudaSuccess || cudaMalloc(&prev, cbytes) != cudaSuccess) {
            cudaFree(Fc);
            GCK(LS_ENOMEM);
        }
        auto restrict_field = [&](const void* bricked, float* out) -> int {
            cudaError_t e = lsk::launch_unpack(bricked, scratch, fine->in0(), 0, s);
            if (e == cudaSuccess) e = lsk::launch_restrict4(scratch, fx, fy, fz, out, s);
            c->launches += 2;
            return e == cudaSuccess ? LS_OK : ls_engine_cuda_fail(e);
        };
        int rr = restrict_field(fine->F, Fc);
        if (!rr) rr = restrict_field(fine->phi[fine->cur], prev);
        for (int j = 0; !rr && j < sp.pairs; ++j) {
            rr = ls_step(fine, 4, sp.cfl * hf, LS_DT_FIXED, 4, nullptr);
            if (rr) break;
            rr = alloc_pair(P);
            if (rr) break;
            rr = restrict_field(fine->phi[fine->cur], P.ref);
            if (rr) { cudaFree(P.phi); cudaFree(P.ref); cudaFree(P.F); break; }
            if (cudaMemcpyAsync(P.phi, prev, cbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(P.F, Fc, cbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(prev, P.ref, cbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
                cudaFree(P.phi); cudaFree(P.ref); cudaFree(P.F);
                rr = LS_ECUDA;
                break;
            }
            L->pairs.push_back(P);
        }
        cudaStreamSynchronize(s);
        cudaFree(Fc);
        cudaFree(prev);
        GCK(rr);
    }
    cudaStreamSynchronize(c->stream);
    ls_destroy(fine);
    cudaFree(scratch);
    return LS_OK;
}

}  // namespace

extern "C" {

int ls_learned_train(ls_ctx* c, const char* pairs_spec, int iters, double lr, double* final_loss)
{
    if (!c || iters < 0 || !(lr > 0)) return LS_EINVAL;
    Spec sp;
    int r = parse_spec(pairs_spec, &sp);
    if (r) return r;
    if (!sp.fine && !(sp.dt > 0.0)) return LS_EINVAL;  // stored pairs: their coarse step is needed
    if (sp.fine) {
        Learned* L = nullptr;
        r = ensure_learned(c, &L);
        if (r) return r;
        if (!L->initialised) return LS_ESTATE;
        r = generate_pairs(c, L, sp);
        if (r) return r;
        if (!(sp.dt > 0.0)) sp.dt = sp.cfl * c->in0().h;  // 4 fine steps of cfl * h / 4
    }
    return ls_learned_train_stored(c, iters, lr, sp.dt, sp.halfwidth, sp.seed, final_loss);
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
                   float* dW, float* db, unsigned* status, void* stream)
{
    if (!x || !dy || !dW || !status || ci < 1 || ci > 16 || co < 1 || co > 16) return LS_EINVAL;
    if (!lsk::conv3_wgrad_shape_ok(nx, ny, nz)) return LS_EINVAL;
    if ((((uintptr_t)x | (uintptr_t)dy) & 15u) != 0) return LS_EINVAL;
    LCK(lsk::launch_conv3_wgrad(x, dy, nx, ny, nz, ci, co, dW, db, status, (cudaStream_t)stream));
    return LS_OK;
}

int ls_learned_features(const float* phi, const float* phit, const float* F, double Fc, double h,
                        long long n, void* X, void* stream)
{
    if (!phi || !phit || !X || n < 1 || !std::isfinite(h) || !(h > 0.0) || !std::isfinite(Fc))
        return LS_EINVAL;
    if (((uintptr_t)X & 15u) != 0) return LS_EINVAL;
    LCK(lsk::launch_features(phi, phit, F, (float)Fc, (float)(1.0 / h), n, X, (cudaStream_t)stream));
    return LS_OK;
}

int ls_learned_loss_grad(const float* z, const float* phi, const float* phit, const float* phiref,
                         long long n, double h, double gamma, void* dz, int* count, double* loss,
                         void* stream)
{
    if (!z || !phi || !phit || !phiref || !dz || !count || !loss || n < 1) return LS_EINVAL;
    if (!std::isfinite(h) || !(h > 0.0) || !std::isfinite(gamma) || !(gamma > 0.0)) return LS_EINVAL;
    if (((uintptr_t)dz & 15u) != 0) return LS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    LCK(cudaMemsetAsync(count, 0, sizeof(int), s));
    LCK(cudaMemsetAsync(loss, 0, sizeof(double), s));
    LCK(lsk::launch_count_mask(phi, gamma, n, count, s));
    LCK(lsk::launch_loss_grad(z, phi, phit, phiref, (float)(1.0 / h), gamma, count, n, dz, loss, s));
    return LS_OK;
}

int ls_adam_step(float* w, const float* g, float* m, float* v, int n, double lr, int step,
                 void* stream)
{
    if (!w || !g || !m || !v || n < 1 || step < 1 || !std::isfinite(lr) || !(lr > 0.0))
        return LS_EINVAL;
    LCK(lsk::launch_adam(w, g, m, v, n, (float)lr, step, (cudaStream_t)stream));
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
