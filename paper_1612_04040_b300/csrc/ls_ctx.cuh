// ls_ctx.cuh -- the context object behind the C ABI (host engine state and
// device buffers), shared by the engine (ls_api.cu) and the learned
// corrector's engine (ls_learned_api.cu).
#pragma once

#include <map>
#include <tuple>
#include <vector>

#include "ls.h"
#include "ls_internal.cuh"

using lsk::Inst;

namespace lsk {
struct Learned;  // corrector state (ls_learned_api.cu)
void learned_free(Learned* L);
struct Output;   // overlapped output (ls_output.cu)
void output_free(Output* O);

// stream-ordered host input/output (ls_stage_inputs, ls_load_staged,
// ls_get_phi_async, ls_wait_host): device staging buffers in row-major
// order, one copy stream per direction, and the events that order them
// against the context's stream
struct HostIO {
    cudaStream_t h2d = nullptr, d2h = nullptr;
    void* in_phi = nullptr;
    void* in_F = nullptr;
    void* out = nullptr;
    cudaEvent_t staged = nullptr;    // h2d: the staged inputs have arrived
    cudaEvent_t consumed = nullptr;  // context stream: ls_load_staged read them
    cudaEvent_t unpacked = nullptr;  // context stream: out holds the result
    cudaEvent_t drained = nullptr;   // d2h: out has been copied to the host
    bool have_phi = false, have_F = false;
};
}  // namespace lsk

namespace lsk {

// host state a captured ls_step graph starts from / leaves behind
struct SchedState {
    int cur = 0;
    int since_rebuild = 0;
    bool band_valid = false;
    bool core_fresh = false;
    int dir = 0;
    bool xface_pending = false;
};

using GraphKey = std::tuple<int, int, int, int, int, int, int, int, long long, int, int, int>;

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    SchedState after;
    unsigned long long launches = 0;
    unsigned long long stencil_launches = 0;
};

}  // namespace lsk

struct ls_ctx {
    int prec = 0;
    size_t esize = 4;
    bool batched = false;
    int n_inst = 1;
    std::vector<Inst> insts;      // host copy of the per-instance parameters
    std::vector<char> inst_phi_set;
    Inst* d_inst = nullptr;       // device copy (batched contexts)
    uint16_t* d_tile_inst = nullptr;  // instance of every global tile (batched)
    uint16_t* d_list_inst = nullptr;  // instance of every list entry (batched)
    int* d_inst_count = nullptr;      // per-instance active counts (batched)
    long long ntiles = 0;
    size_t npts = 0;
    size_t max_inst_pts = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;  // used for graph capture when stream is NULL
    void* phi[2] = {nullptr, nullptr};
    int cur = 0;
    void* F = nullptr;            // bricked speed field (lazy)
    void* tile_maxF = nullptr;    // per-tile max |F| (lazy)
    uint8_t* tile_sgn = nullptr;  // per-tile sign code of a speed field (lazy)
    void* staging = nullptr;      // row-major staging buffer (lazy)
    void* snapshot = nullptr;     // ls_snapshot copy of phi (lazy)
    double* init_params = nullptr;  // device copy of Step 0 shape / speed parameters
    int init_params_cap = 0;
    uint8_t* core = nullptr;
    uint8_t* act = nullptr;       // bit 0: active, bit 1: active before the last rebuild
    uint8_t* mark = nullptr;      // new-active marks of the incremental rebuild (0 between)
    int* d_leave = nullptr;       // ids of the tiles leaving the set at an incremental rebuild
    int* d_nleave = nullptr;
    int* list = nullptr;
    uint8_t* list_info = nullptr;
    int* d_count = nullptr;
    unsigned* d_done = nullptr;   // last-block counters: dilate, scatter, N-flag count
    int* block_counts = nullptr;
    int nblocks = 0;
    int* d_rowcnt = nullptr;      // per tile row active counts (slab split, lazy)
    lsk::StepScalars* d_sc = nullptr;
    unsigned long long* d_Mbits = nullptr;
    unsigned long long* d_updates = nullptr;
    unsigned long long* d_updates2 = nullptr;  // points of two-step passes
    unsigned* d_status = nullptr;
    unsigned* h_nonfinite = nullptr;  // pack's non-finite flag: page-locked host word
    unsigned* d_nonfinite = nullptr;  // the same word as the kernels address it
    // host-side state
    bool band_valid = false;
    bool core_fresh = false;
    bool full_domain = false;
    bool have_halfwidth = false;
    double halfwidth = 0.0;
    int since_rebuild = 0;
    int dir = 0;                  // traversal direction of the next stencil launch
    int dilation = 26;            // band dilation: 26 or 6 face neighbours
    int rebuild_mode = 0;         // LS_REBUILD_AUTO / _FULL / _INCREMENTAL
    int dt_mode = LS_DT_FIXED;
    double dt_value = 0.0;
    lsk::StepConfig cfg;
    // graphs
    bool use_graphs = false;
    std::map<lsk::GraphKey, lsk::GraphEntry> graphs;
    // profiling
    unsigned long long launches = 0;
    unsigned long long stencil_launches = 0;
    bool profiling = false;
    double stencil_ms = 0.0;
    unsigned long long stencil_timed = 0;
    std::vector<cudaEvent_t> ev_free;
    double reinit_ms = 0.0;
    unsigned long long reinit_timed = 0;
    struct EvPair { cudaEvent_t e0, e1; bool reinit; int count; };
    std::vector<EvPair> ev_pending;
    bool ev_open = false;          // an event run of stencil launches is open
    bool ev_skip = false;          // the open run is not timed (sampled profile)
    int prof_every = 1;            // time one run of stencil launches in prof_every
    unsigned long long prof_runs = 0;        // runs opened since profiling was enabled
    unsigned long long* d_updates_timed = nullptr;  // updates of the timed launches
    int ev_open_kind = 0;          // 0 plain / advance, 1 reinitialisation
    int ev_open_n = 0;             // launches in the open run
    cudaEvent_t ev_open_e0 = nullptr;

    // local scheme (section 1.1, Steps 1-3)
    int scheme = LS_SCHEME_PLAIN;
    double beta_in_h = 0.0;
    double dtau_in_h = 0.5;
    int reinit_iters = -1;
    uint32_t* nmask = nullptr;                 // N bits, 16 words per list entry
    uint8_t* list_nact = nullptr;              // active face neighbours per list entry
    float* xface = nullptr;                    // frozen x-face copies per tile (FP32 single grid)
    bool xface_pending = false;                // some copy of the current band is unwritten
    uint8_t* nflag = nullptr;                  // per list entry: the tile holds a point of N
    int* nl = nullptr;                         // tiles holding N points (ascending) ...
    uint8_t* nl_info = nullptr;                // ... their info bytes ...
    uint32_t* nmask2 = nullptr;                // ... and N bits
    int* d_ncount = nullptr;                   // their number
    unsigned long long* d_rupdates = nullptr;  // reinitialisation point-iterations
    unsigned long long* d_breaches = nullptr;

    // overlapped output
    lsk::Output* output = nullptr;
    lsk::HostIO* hio = nullptr;
    int output_every = 0;
    long long step_count = 0;     // steps taken over the context's lifetime

    // learned corrector
    int step_mode = LS_PLAIN;
    lsk::Learned* learned = nullptr;

    Inst& in0() { return insts[0]; }
    const Inst* dinst() const { return batched ? d_inst : nullptr; }
    const uint16_t* tinst() const { return batched ? d_tile_inst : nullptr; }
};


// engine helpers used by the learned corrector's engine
int ls_engine_cuda_fail(cudaError_t e);
int ls_engine_pack(ls_ctx* c, const Inst& in, const void* src, int on_device, void* dst);
int ls_engine_learned_after_step(ls_ctx* c, cudaStream_t s);
int ls_engine_output_after_step(ls_ctx* c, cudaStream_t s);
