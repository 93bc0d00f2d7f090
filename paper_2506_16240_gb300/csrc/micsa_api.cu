// micsa_api.cu -- host side of the C ABI declared in include/micsa.h: argument
// checking, device memory of a handle, the refresh cut points (host FP64) and
// the launch sequence of a run (Sec. 2.8 procedure with gamma = 1).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include "micsa_internal.h"
#include "../../include/micsa.h"

using namespace micsa;

struct micsa_ctx {
    int L = 0, S = 0, R = 0;
    int gamma = 1;       // daemons (or walkers) per spin; a timestep is gamma sweeps
    int walkers = 0;     // walkers wander after every timestep (Sec. 2.6)
    uint64_t seed = 0;
    int64_t t = 0;
    Geometry geo{};
    int device = 0;
    int8_t *d_spins = nullptr;
    uint8_t *d_daemons = nullptr;
    uint8_t *d_bonds = nullptr;
    unsigned long long *d_meas = nullptr;
    uint8_t *d_stage = nullptr;  // natural-layout staging for state / coupling copies
    unsigned long long *d_first = nullptr;  // first invalid byte of a staged copy
    size_t stage_bytes = 0;
    size_t device_bytes = 0;
    int64_t launches = 0;  // kernels launched by this handle
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;  // graphs are captured here (never the legacy stream)
    int sm_count = 0;
    LaunchConfig lc;                // requested launch shape
    int blocks_per_sm = -1;         // -1: resident capacity (grid-stride), 0: no cap
    // per-run sweep parameter table: pinned host copy, device copy
    SweepParam *h_params = nullptr;
    SweepParam *d_params = nullptr;
    int64_t params_cap = 0;
    cudaEvent_t params_free = nullptr;  // the last upload of h_params has been consumed
    int64_t *d_cursor = nullptr;
    cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};  // [kind]: G sweeps + cursor advance
    int engine = MICSA_ENGINE_AUTO;  // which kernel runs MicSA sweeps
    int resident_sweeps = 256;       // sweeps per resident launch
    ResidentUnit *d_units = nullptr; // one unit per (sample, replica)
    int graph_g[3] = {0, 0, 0};
    int64_t graph_kernels[3] = {0, 0, 0};  // kernels per replay of each graph
    int chains = 1;                  // replica groups captured as concurrent chains
    cudaStream_t aux_stream[3] = {nullptr, nullptr, nullptr};  // capture streams of chains 1..3
    cudaEvent_t fork_ev = nullptr, join_ev[3] = {nullptr, nullptr, nullptr};
    uint32_t *d_planes = nullptr;    // multispin planes [S*R][3][2][L^3/64] (MULTISPIN_GLOBAL)
    uint32_t *d_bplanes = nullptr;   // bond planes [S][6][2][L^3/64]
    int msg_rpt = 0;                 // replicas per thread of MULTISPIN_GLOBAL (0: automatic)
    OnchipPlan oc;                   // partition of the ONCHIP engine (oc.grid == 0: not planned)
    int16_t *d_oc_nbrs = nullptr;    // its neighbour table
    unsigned *d_oc_flags = nullptr;  // its epoch flags
    int *d_error = nullptr;          // device-side wait time-outs (ONCHIP, TMA)
    TmaMaps tma;                     // tensor maps of the TMA engine (tma.valid: encoded)
    int tma_ctas = 0;                // its persistent grid
    long long wait_limit = 1ll << 22;  // polls per wait
    std::string err;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int fail(micsa_t h, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(micsa_t h, int code, const char *fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return code;
}

int cuda_fail(micsa_t h, cudaError_t e, const char *what) {
    return fail(h, e == cudaErrorMemoryAllocation ? MICSA_E_OOM : MICSA_E_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CK(h, expr, what)                                    \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

int64_t sites(const micsa_ctx *h) { return (int64_t)h->L * h->L * h->L; }

uint64_t cut_point(double c) {
    const double v = std::floor(c * 4294967296.0);
    if (v >= 4294967296.0) return 4294967296ull;
    if (v <= 0.0) return 0;
    return (uint64_t)v;
}

bool temperature_ok(double T) { return T > 0.0 && std::isfinite(T); }

int ensure_stage(micsa_t h, size_t bytes) {
    if (h->stage_bytes >= bytes) return MICSA_OK;
    if (h->d_stage) {
        CK(h, cudaStreamSynchronize(h->stream), "synchronize before staging realloc");
        cudaFree(h->d_stage);
        h->device_bytes -= h->stage_bytes;
        h->d_stage = nullptr;
        h->stage_bytes = 0;
    }
    CK(h, cudaMalloc(&h->d_stage, bytes), "cudaMalloc staging");
    h->stage_bytes = bytes;
    h->device_bytes += bytes;
    return MICSA_OK;
}

// Index of the first invalid byte of n staged bytes at dev (mode 0: +-1,
// mode 1: 0..3) in *first, -1 if there is none; checked on the device, so that
// a caller's buffer is read once (by the copy) and the state is untouched when
// it is rejected.
int staged_first_invalid(micsa_t h, const uint8_t *dev, int64_t n, int mode, int64_t *first) {
    if (!h->d_first) {
        CK(h, cudaMalloc(&h->d_first, sizeof(unsigned long long)), "cudaMalloc check word");
        h->device_bytes += sizeof(unsigned long long);
    }
    CK(h, launch_first_invalid(dev, n, mode, h->d_first, h->stream), "validate staged bytes");
    ++h->launches;
    unsigned long long v = 0;
    CK(h, cudaMemcpyAsync(&v, h->d_first, sizeof v, cudaMemcpyDeviceToHost, h->stream), "read check word");
    CK(h, cudaStreamSynchronize(h->stream), "validate synchronize");
    *first = v == ~0ull ? -1 : (int64_t)v;
    return MICSA_OK;
}

SweepArgs sweep_args(const micsa_ctx *h) {
    SweepArgs a{};
    a.spins = h->d_spins;
    a.daemons = h->d_daemons;
    a.bonds = h->d_bonds;
    a.geo = h->geo;
    a.S = h->S;
    a.R = h->R;
    a.gamma = h->gamma;
    a.key0 = (uint32_t)(h->seed & 0xFFFFFFFFu);
    a.key1 = (uint32_t)(h->seed >> 32);
    a.r0 = 0;
    a.r1 = h->R;
    return a;
}

// Replicas [r0, r1) of replica group c of n (as even as possible).
void replica_group(const micsa_ctx *h, int c, int n, int &r0, int &r1) {
    r0 = c * h->R / n;
    r1 = (c + 1) * h->R / n;
}

void drop_graphs(micsa_t h) {
    for (int i = 0; i < 3; ++i) {
        if (h->graph[i]) cudaGraphExecDestroy(h->graph[i]);
        h->graph[i] = nullptr;
        h->graph_g[i] = 0;
    }
}

// Effective launch shape for this handle: vector width the pitch allows and the
// grid cap of the grid-stride loop.
LaunchConfig effective_config(micsa_t h, bool metro) {
    LaunchConfig lc = h->lc;
    lc.nw = vector_words(h->geo, lc.nw);
    if (h->blocks_per_sm < 0) {
        const dim3 b = block_shape(h->R, lc.regcap && lc.block > 128 ? 128 : lc.block, lc.regcap ? 128 : 256);
        const bool full = !metro && h->geo.P == h->geo.Lh;
        const int per_sm = lc.pairs && full  ? max_resident_blocks_pairs(lc.nw, (int)(b.x * b.y))
                           : lc.reps && full ? max_resident_blocks_reps(lc.nw, lc.block)
                                             : max_resident_blocks(metro, lc.nw, (int)(b.x * b.y), lc.regcap);
        lc.max_blocks = per_sm > 0 ? per_sm * h->sm_count : 0;
    } else {
        lc.max_blocks = h->blocks_per_sm * h->sm_count;
    }
    return lc;
}

int ensure_params(micsa_t h, int64_t n) {
    if (h->params_cap >= n) {
        CK(h, cudaEventSynchronize(h->params_free), "wait for the previous parameter upload");
        return MICSA_OK;
    }
    CK(h, cudaStreamSynchronize(h->stream), "synchronize before parameter realloc");
    cudaFreeHost(h->h_params);
    cudaFree(h->d_params);
    h->h_params = nullptr;
    h->d_params = nullptr;
    h->device_bytes -= sizeof(SweepParam) * (size_t)h->params_cap;
    h->params_cap = 0;
    drop_graphs(h);  // captured graphs point at the old table
    int64_t cap = 1024;
    while (cap < n) cap *= 2;
    CK(h, cudaMallocHost(&h->h_params, sizeof(SweepParam) * (size_t)cap), "cudaMallocHost parameters");
    CK(h, cudaMalloc(&h->d_params, sizeof(SweepParam) * (size_t)cap), "cudaMalloc parameters");
    h->params_cap = cap;
    h->device_bytes += sizeof(SweepParam) * (size_t)cap;
    return MICSA_OK;
}

enum GraphKind { kGraphMicsa = 0, kGraphMetro = 1, kGraphPlanes = 2 };

int msg_rpt(const micsa_ctx *h, int nw, int n_rep) {
    return h->msg_rpt > 0 ? h->msg_rpt : msg_default_rpt(h->geo, h->S, n_rep, nw, h->sm_count);
}

// One half-sweep of the bit-plane engine over replicas [r0, r1), reading
// params[*cursor + k].
cudaError_t launch_planes_half(micsa_t h, const LaunchConfig &lc, int parity, const int64_t *cursor, int64_t k,
                               int r0, int r1, cudaStream_t st, bool metro = false) {
    return launch_msg_half(h->d_planes, h->d_bplanes, h->geo, h->S, h->R, r0, r1, msg_rpt(h, lc.nw, r1 - r0), lc.nw,
                           lc.regcap, parity, h->gamma, h->walkers, (uint32_t)(h->seed & 0xFFFFFFFFu), (uint32_t)(h->seed >> 32),
                           h->d_params, cursor, k, lc.pdl, st, metro);
}

// One timestep of the bit-plane engine for replicas [r0, r1): gamma sweeps
// (table entries k*gamma + alpha). With walkers the wandering step of the
// previous timestep is applied by these half-sweeps as they read their daemons
// (the table's gather flag); the last one of a run by run_planes.
cudaError_t launch_planes_timestep(micsa_t h, const LaunchConfig &lc, const int64_t *cursor, int64_t k, int r0,
                                   int r1, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    for (int al = 0; al < h->gamma && e == cudaSuccess; ++al)
        for (int p = 0; p < 2 && e == cudaSuccess; ++p)
            e = launch_planes_half(h, lc, p, cursor, k * h->gamma + al, r0, r1, st);
    return e;
}

int64_t planes_timestep_kernels(const micsa_ctx *h) { return 2 * (int64_t)h->gamma; }

// One half-sweep of graph kind gi over replica group c of `chains`.
cudaError_t launch_group_half(micsa_t h, int gi, const LaunchConfig &lc, SweepArgs a, int c, int chains,
                              cudaStream_t st) {
    replica_group(h, c, chains, a.r0, a.r1);
    if (gi == kGraphPlanes) return launch_planes_half(h, lc, a.parity, a.cursor, a.k, a.r0, a.r1, st);
    if (gi == kGraphMicsa && h->engine == MICSA_ENGINE_TMA && h->tma.valid)
        return launch_tma_half(h->tma, h->d_spins, h->d_daemons, h->geo, h->S, h->R, a.r0, a.r1, a.parity, a.key0,
                               a.key1, a.params, a.cursor, a.k, h->d_error, h->wait_limit, h->tma_ctas, lc.pdl, st);
    return launch_half_sweep(a, gi == kGraphMetro, lc, st);
}

// Capture G sweeps (2G half-sweeps reading params[*cursor + k]) and the cursor
// advance into an executable graph. With chains > 1 the replica groups are
// independent chains of half-sweeps on forked capture streams (they touch
// disjoint replicas), joined before the cursor advance, so that one chain's
// launch gap and tail overlap the other chains' work.
int capture_graph(micsa_t h, int gi, int G, const LaunchConfig &lc) {
    if (h->graph[gi] && h->graph_g[gi] == G) return MICSA_OK;
    if (h->graph[gi]) cudaGraphExecDestroy(h->graph[gi]);
    h->graph[gi] = nullptr;
    const int chains = std::min(h->chains, h->R);
    for (int c = 1; c < chains; ++c) {
        if (!h->aux_stream[c - 1])
            CK(h, cudaStreamCreateWithFlags(&h->aux_stream[c - 1], cudaStreamNonBlocking), "cudaStreamCreate");
        if (!h->join_ev[c - 1])
            CK(h, cudaEventCreateWithFlags(&h->join_ev[c - 1], cudaEventDisableTiming), "cudaEventCreate");
    }
    if (!h->fork_ev) CK(h, cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming), "cudaEventCreate");
    SweepArgs a = sweep_args(h);
    a.params = h->d_params;
    a.cursor = h->d_cursor;
    CK(h, cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = cudaSuccess;
    if (chains > 1) {
        e = cudaEventRecord(h->fork_ev, h->capture_stream);
        for (int c = 1; c < chains && e == cudaSuccess; ++c) e = cudaStreamWaitEvent(h->aux_stream[c - 1], h->fork_ev, 0);
    }
    for (int c = 0; c < chains && e == cudaSuccess; ++c) {
        cudaStream_t st = c == 0 ? h->capture_stream : h->aux_stream[c - 1];
        if (gi == kGraphPlanes) {  // G timesteps
            int r0, r1;
            replica_group(h, c, chains, r0, r1);
            for (int k = 0; k < G && e == cudaSuccess; ++k) e = launch_planes_timestep(h, lc, h->d_cursor, k, r0, r1, st);
            continue;
        }
        for (int k = 0; k < G && e == cudaSuccess; ++k)
            for (int p = 0; p < 2 && e == cudaSuccess; ++p) {
                a.k = k;
                a.parity = p;
                e = launch_group_half(h, gi, lc, a, c, chains, st);
            }
    }
    for (int c = 1; c < chains && e == cudaSuccess; ++c) {
        e = cudaEventRecord(h->join_ev[c - 1], h->aux_stream[c - 1]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->capture_stream, h->join_ev[c - 1], 0);
    }
    const int64_t step = gi == kGraphPlanes ? (int64_t)G * h->gamma : G;
    if (e == cudaSuccess) e = launch_advance_cursor(h->d_cursor, step, lc.pdl, h->capture_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->capture_stream, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(h, e, "launch during capture");
    }
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "end capture");
    e = cudaGraphInstantiate(&h->graph[gi], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        h->graph[gi] = nullptr;
        return cuda_fail(h, e, "graph instantiate");
    }
    h->graph_g[gi] = G;
    h->graph_kernels[gi] = (gi == kGraphPlanes ? planes_timestep_kernels(h) : 2) * (int64_t)G * chains + 1;
    return MICSA_OK;
}

// The engine a MicSA run uses now.
int active_engine(micsa_t h) {
    if (h->engine == MICSA_ENGINE_MULTISPIN_GLOBAL)  // gamma families and walkers included
        return msg_supported(h->geo) ? MICSA_ENGINE_MULTISPIN_GLOBAL : MICSA_ENGINE_STREAM;
    if (h->engine == MICSA_ENGINE_STREAM || h->gamma > 1 || h->walkers) return MICSA_ENGINE_STREAM;
    if (h->engine == MICSA_ENGINE_ONCHIP) return h->oc.grid > 0 ? MICSA_ENGINE_ONCHIP : MICSA_ENGINE_STREAM;
    if (h->engine == MICSA_ENGINE_TMA) return h->tma.valid ? MICSA_ENGINE_TMA : MICSA_ENGINE_STREAM;
    if (!h->d_units) return MICSA_ENGINE_STREAM;
    if (h->engine == MICSA_ENGINE_RESIDENT) return MICSA_ENGINE_RESIDENT;
    if (multispin_smem_bytes(h->geo) > 0) return MICSA_ENGINE_MULTISPIN;
    return h->engine == MICSA_ENGINE_MULTISPIN ? MICSA_ENGINE_STREAM : MICSA_ENGINE_RESIDENT;
}

bool use_resident(micsa_t h) {
    const int e = active_engine(h);
    return e == MICSA_ENGINE_RESIDENT || e == MICSA_ENGINE_MULTISPIN;
}

// Device memory of the bit-plane engine, allocated on first use.
int ensure_planes(micsa_t h) {
    if (h->d_planes) return MICSA_OK;
    const size_t WP = (size_t)msg_plane_words(h->geo);
    const size_t state =
        sizeof(uint32_t) * (size_t)h->S * h->R * (size_t)msg_planes_per_replica(h->gamma, h->walkers) * WP;
    const size_t bonds = sizeof(uint32_t) * (size_t)h->S * 12 * WP;
    CK(h, cudaMalloc(&h->d_planes, state), "cudaMalloc planes");
    cudaError_t e = cudaMalloc(&h->d_bplanes, bonds);
    if (e != cudaSuccess) {
        cudaFree(h->d_planes);
        h->d_planes = nullptr;
        return cuda_fail(h, e, "cudaMalloc bond planes");
    }
    h->device_bytes += state + bonds;
    return MICSA_OK;
}

// MicSA timesteps [0, n) of the uploaded table (n * gamma entries) on bit
// planes in HBM: bytes -> planes, whole blocks of G timesteps by graph replay,
// the rest directly, planes -> bytes. A timestep is gamma sweeps (each the even
// half-sweep followed by the odd one) and, with walkers, the wandering step.
int run_planes(micsa_t h, int64_t n, const LaunchConfig &lc, bool metro = false) {
    if (int rc = ensure_planes(h)) return rc;
    const int buf0 = h->walkers ? (int)(h->t & 1) : 0, buf1 = h->walkers ? (int)((h->t + n) & 1) : 0;
    CK(h, msg_convert(h->d_planes, h->d_bplanes, h->d_spins, h->d_daemons, h->d_bonds, h->geo, h->S, h->R, h->gamma,
                      h->walkers, buf0, true, h->stream), "convert to planes");
    h->launches += 2;
    const int G = metro ? 0 : lc.graph_sweeps;  // Metropolis sweeps: direct launches
    int64_t done = 0;
    if (G > 0 && n >= 2 * (int64_t)G) {
        if (int rc = capture_graph(h, kGraphPlanes, G, lc)) return rc;
        CK(h, cudaMemsetAsync(h->d_cursor, 0, sizeof(int64_t), h->stream), "reset cursor");
        const int64_t reps = n / G;
        for (int64_t r = 0; r < reps; ++r) CK(h, cudaGraphLaunch(h->graph[kGraphPlanes], h->stream), "graph launch");
        h->launches += reps * h->graph_kernels[kGraphPlanes];
        done = reps * G;
    }
    for (int64_t k = done; k < n; ++k) {
        if (metro) {  // one sweep per timestep (gamma 1)
            for (int p = 0; p < 2; ++p)
                CK(h, launch_planes_half(h, lc, p, nullptr, k, 0, h->R, h->stream, true), "plane Metropolis launch");
            h->launches += 2;
            continue;
        }
        CK(h, launch_planes_timestep(h, lc, nullptr, k, 0, h->R, h->stream), "plane timestep launch");
        h->launches += planes_timestep_kernels(h);
    }
    if (h->walkers) {  // the wandering step after the run's last timestep
        CK(h, launch_msg_wander(h->d_planes, h->geo, h->S, h->R, 0, h->R, h->gamma, h->d_params, nullptr,
                                (n - 1) * h->gamma, lc.pdl, h->stream), "wander launch");
        ++h->launches;
    }
    CK(h, msg_convert(h->d_planes, nullptr, h->d_spins, h->d_daemons, nullptr, h->geo, h->S, h->R, h->gamma,
                      h->walkers, buf1, false, h->stream), "convert from planes");
    ++h->launches;
    return MICSA_OK;
}

// MicSA sweeps [0, n) of the uploaded table with the shared-memory resident
// kernel, resident_sweeps per launch; every (sample, replica) is one unit.
int run_resident(micsa_t h, int64_t n, const LaunchConfig &lc) {
    const bool ms = active_engine(h) == MICSA_ENGINE_MULTISPIN;
    const size_t smem = ms ? multispin_smem_bytes(h->geo) : resident_smem_bytes(h->geo);
    const int per_sm = ms ? multispin_blocks_per_sm(false, smem) : resident_blocks_per_sm(false, smem);
    const int n_units = h->S * h->R;
    int grid = (per_sm > 0 ? per_sm : 1) * h->sm_count;
    if (grid > n_units) grid = n_units;
    ResidentArgs ra{};
    ra.units = h->d_units;
    ra.n_units = n_units;
    ra.geo = h->geo;
    ra.key0 = (uint32_t)(h->seed & 0xFFFFFFFFu);
    ra.key1 = (uint32_t)(h->seed >> 32);
    ra.params = h->d_params;
    for (int64_t k0 = 0; k0 < n; k0 += h->resident_sweeps) {
        ra.k0 = k0;
        ra.K = (int)std::min<int64_t>(h->resident_sweeps, n - k0);
        if (ms)
            CK(h, launch_multispin(ra, false, smem, grid, lc.pdl, h->stream), "multispin launch");
        else
            CK(h, launch_resident(ra, false, smem, grid, lc.pdl, h->stream), "resident launch");
        ++h->launches;
    }
    return MICSA_OK;
}

int ensure_error_word(micsa_t h) {
    if (h->d_error) return MICSA_OK;
    CK(h, cudaMalloc(&h->d_error, sizeof(int)), "cudaMalloc error word");
    CK(h, cudaMemset(h->d_error, 0, sizeof(int)), "clear error word");
    return MICSA_OK;
}

// Tensor maps and grid of the TMA engine.
int plan_tma(micsa_t h) {
    if (h->tma.valid) return MICSA_OK;
    if (!tma_supported(h->geo, h->gamma, h->walkers) || tma_stages(h->geo) < 2)
        return fail(h, MICSA_E_INVALID_ARG, "the TMA engine needs L %% 8 == 0, a row pitch of 16..256 bytes in "
                                            "steps of 16, gamma = 1 and no walkers (L=%d)", h->L);
    if (int rc = ensure_error_word(h)) return rc;
    const int ctas = tma_max_ctas(h->geo, h->sm_count);
    if (ctas < 1) return fail(h, MICSA_E_CUDA, "the TMA kernel cannot be resident");
    CK(h, tma_encode(h->tma, h->d_spins, h->d_daemons, h->d_bonds, h->geo, h->S, h->R), "encode tensor maps");
    h->tma_ctas = ctas;
    return MICSA_OK;
}

// Partition, neighbour table and flags of the ONCHIP engine for words-per-item nw.
int plan_onchip(micsa_t h, int nw) {
    if (h->oc.grid > 0 && h->oc.nw == nw) return MICSA_OK;
    OnchipPlan plan;
    if (h->gamma > 1 || h->walkers || !onchip_plan(h->geo, h->S, h->R, h->sm_count, nw, plan))
        return fail(h, MICSA_E_INVALID_ARG, "the on-chip engine does not fit this lattice (L=%d S=%d R=%d)", h->L,
                    h->S, h->R);
    CK(h, cudaStreamSynchronize(h->stream), "synchronize before planning");
    cudaFree(h->d_oc_nbrs);
    cudaFree(h->d_oc_flags);
    h->d_oc_nbrs = nullptr;
    h->d_oc_flags = nullptr;
    h->oc = OnchipPlan();
    CK(h, cudaMalloc(&h->d_oc_nbrs, sizeof(int16_t) * plan.table.size()), "cudaMalloc neighbour table");
    CK(h, cudaMemcpy(h->d_oc_nbrs, plan.table.data(), sizeof(int16_t) * plan.table.size(), cudaMemcpyHostToDevice),
       "upload neighbour table");
    CK(h, cudaMalloc(&h->d_oc_flags, sizeof(unsigned) * onchip_flag_words(plan.grid)), "cudaMalloc flags");
    if (int rc = ensure_error_word(h)) return rc;
    h->oc = std::move(plan);
    return MICSA_OK;
}

// MicSA sweeps [0, n) of the uploaded table with the on-chip engine,
// resident_sweeps sweeps per cooperative launch.
int run_onchip(micsa_t h, int64_t n, const LaunchConfig &lc) {
    if (int rc = plan_onchip(h, lc.nw)) return rc;
    for (int64_t k0 = 0; k0 < n; k0 += h->resident_sweeps) {
        const int K = (int)std::min<int64_t>(h->resident_sweeps, n - k0);
        CK(h, launch_onchip(h->oc, h->d_spins, h->d_daemons, h->d_bonds, h->geo, h->S, h->R,
                            (uint32_t)(h->seed & 0xFFFFFFFFu), (uint32_t)(h->seed >> 32), h->d_params, k0, K,
                            h->d_oc_flags, h->d_error, h->d_oc_nbrs, h->wait_limit, h->stream),
           "on-chip launch");
        ++h->launches;
    }
    return MICSA_OK;
}

// A device-side wait that ran out since the last check (ONCHIP engine).
int check_device_error(micsa_t h) {
    if (!h->d_error) return MICSA_OK;
    int v = 0;
    CK(h, cudaMemcpyAsync(&v, h->d_error, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "read error word");
    CK(h, cudaStreamSynchronize(h->stream), "synchronize error word");
    if (v) {
        CK(h, cudaMemsetAsync(h->d_error, 0, sizeof(int), h->stream), "clear error word");
        return fail(h, MICSA_E_TIMEOUT, "a device-side wait of the on-chip engine ran out; the state is not valid");
    }
    return MICSA_OK;
}

// Upload the table of n sweeps and run them: whole blocks of G sweeps by graph
// replay, the rest by direct launches. Every sweep is the even half-sweep
// followed by the odd one (Sec. 2.8 steps (i), (ii)).
int run_table(micsa_t h, bool metro, int64_t n) {
    if (n == 0) return MICSA_OK;
    const LaunchConfig lc = effective_config(h, metro);
    CK(h, cudaMemcpyAsync(h->d_params, h->h_params, sizeof(SweepParam) * (size_t)n,
                          cudaMemcpyHostToDevice, h->stream), "upload sweep parameters");
    CK(h, cudaEventRecord(h->params_free, h->stream), "record parameter event");
    if (!metro && use_resident(h)) return run_resident(h, n, lc);
    // bit planes: MicSA, and Metropolis with one daemon family and no walkers (a
    // timestep is then one sweep; the daemon planes ride along unchanged)
    if (active_engine(h) == MICSA_ENGINE_MULTISPIN_GLOBAL && (!metro || (h->gamma == 1 && !h->walkers)))
        return run_planes(h, n, lc, metro);
    if (!metro && active_engine(h) == MICSA_ENGINE_ONCHIP) return run_onchip(h, n, lc);
    const int G = lc.graph_sweeps;
    int64_t done = 0;
    if (G > 0 && n >= 2 * (int64_t)G) {
        if (int rc = capture_graph(h, metro ? kGraphMetro : kGraphMicsa, G, lc)) return rc;
        CK(h, cudaMemsetAsync(h->d_cursor, 0, sizeof(int64_t), h->stream), "reset cursor");
        const int64_t reps = n / G;
        for (int64_t r = 0; r < reps; ++r)
            CK(h, cudaGraphLaunch(h->graph[metro ? 1 : 0], h->stream), "graph launch");
        h->launches += reps * h->graph_kernels[metro ? 1 : 0];
        done = reps * G;
    }
    SweepArgs a = sweep_args(h);
    a.params = h->d_params;
    a.cursor = nullptr;
    for (int64_t k = done; k < n; ++k)
        for (int p = 0; p < 2; ++p) {
            a.k = k;
            a.parity = p;
            CK(h, launch_group_half(h, metro ? kGraphMetro : kGraphMicsa, lc, a, 0, 1, h->stream), "half-sweep launch");
            ++h->launches;
        }
    return MICSA_OK;
}

bool schedule_ok(micsa_t h, const double *schedule, int64_t n_sweeps) {
    if (n_sweeps < 0 || (n_sweeps > 0 && !schedule)) {
        fail(h, MICSA_E_INVALID_ARG, "n_sweeps must be >= 0 and schedule non-NULL");
        return false;
    }
    for (int64_t k = 0; k < n_sweeps; ++k)
        if (!temperature_ok(schedule[k])) {
            fail(h, MICSA_E_INVALID_ARG, "schedule[%lld] = %g is not a finite T > 0", (long long)k,
                 schedule[k]);
            return false;
        }
    return true;
}

// Couplings and spins from the seed (Sec. 2.1 and the disordered start of
// Sec. 3), daemons zero, t = 0.
int init_from_seed(micsa_t h, uint64_t seed) {
    const size_t state = (size_t)h->S * h->R * h->gamma * 2 * h->geo.half;
    const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
    h->seed = seed;
    CK(h, cudaMemsetAsync(h->d_daemons, 0, state, h->stream), "memset daemons");
    CK(h, launch_init_couplings(h->d_bonds, h->geo, h->S, k0, k1, h->stream), "init couplings");
    CK(h, launch_init_spins(h->d_spins, h->geo, h->S, h->R, k0, k1, h->stream), "init spins");
    h->launches += 2;
    h->t = 0;
    return MICSA_OK;
}

// Timesteps with gamma daemon families or walkers (Sec. 2.8): sweep alpha of
// timestep k is table entry k * gamma + alpha; walkers wander after the last
// sweep of each timestep. Direct launches.
int run_families(micsa_t h, int64_t n_steps, const LaunchConfig &lc) {
    SweepArgs a = sweep_args(h);
    a.params = h->d_params;
    a.cursor = nullptr;
    for (int64_t k = 0; k < n_steps; ++k) {
        for (int al = 0; al < h->gamma; ++al)
            for (int p = 0; p < 2; ++p) {
                a.k = k * h->gamma + al;
                a.parity = p;
                CK(h, launch_half_sweep(a, false, lc, h->stream), "half-sweep launch");
                ++h->launches;
            }
        if (h->walkers) {
            const int parity = (int)((h->t + k) & 1);
            CK(h, launch_wander(h->d_daemons, h->geo, (int64_t)h->S * h->R, h->gamma, parity, h->stream),
               "wander launch");
            ++h->launches;
        }
    }
    return MICSA_OK;
}

// MicSA run of n_steps timesteps with refresh before timestep t iff
// is_refresh(t) (Sec. 2.7, 2.8); a timestep is gamma sweeps.
template <class IsRefresh>
int run_micsa(micsa_t h, const double *schedule, int64_t n_sweeps, IsRefresh is_refresh) {
    if (!h) return MICSA_E_INVALID_ARG;
    if (!schedule_ok(h, schedule, n_sweeps)) return MICSA_E_INVALID_ARG;
    if (n_sweeps == 0) return MICSA_OK;
    DeviceGuard dg(h->device);
    const int G = h->gamma;
    if (int rc = ensure_params(h, n_sweeps * G)) return rc;
    double last_T = -1.0;
    uint64_t th[3] = {0, 0, 0};
    for (int64_t k = 0; k < n_sweeps; ++k) {
        const int64_t t = h->t + k;
        const int mode = is_refresh(t) ? kModeRefresh : kModeMicsa;
        if (mode == kModeRefresh && schedule[k] != last_T) {
            micsa_daemon_thresholds(schedule[k], th);
            last_T = schedule[k];
        }
        const bool gather = h->walkers && k > 0 && active_engine(h) == MICSA_ENGINE_MULTISPIN_GLOBAL;
        for (int al = 0; al < G; ++al) {
            SweepParam &q = h->h_params[k * G + al];
            q.t = t;
            q.mode = mode;
            q.th0 = th[0];
            q.th1 = th[1];
            q.th2 = th[2];
            q.alpha = al;
            q.gather = gather ? 1 : 0;
            q.reserved = 0;
        }
    }
    if (G == 1 && !h->walkers) {
        if (int rc = run_table(h, false, n_sweeps)) return rc;
    } else if (active_engine(h) == MICSA_ENGINE_MULTISPIN_GLOBAL) {
        const LaunchConfig lc = effective_config(h, false);
        CK(h, cudaMemcpyAsync(h->d_params, h->h_params, sizeof(SweepParam) * (size_t)(n_sweeps * G),
                              cudaMemcpyHostToDevice, h->stream), "upload sweep parameters");
        CK(h, cudaEventRecord(h->params_free, h->stream), "record parameter event");
        if (int rc = run_planes(h, n_sweeps, lc)) return rc;
    } else {
        const LaunchConfig lc = effective_config(h, false);
        CK(h, cudaMemcpyAsync(h->d_params, h->h_params, sizeof(SweepParam) * (size_t)(n_sweeps * G),
                              cudaMemcpyHostToDevice, h->stream), "upload sweep parameters");
        CK(h, cudaEventRecord(h->params_free, h->stream), "record parameter event");
        if (int rc = run_families(h, n_sweeps, lc)) return rc;
    }
    h->t += n_sweeps;
    return MICSA_OK;
}

}  // namespace

extern "C" {

int micsa_daemon_thresholds(double T, uint64_t theta[3]) {
    if (!theta || !temperature_ok(T)) return MICSA_E_INVALID_ARG;
    const double beta = 1.0 / T;
    const double x = std::exp(-4.0 * beta);
    double p0;
    if (x == 1.0) {
        p0 = 0.25;
    } else {
        const double x2 = x * x;
        const double x4 = x2 * x2;
        p0 = (1.0 - x) / (1.0 - x4);
    }
    const double p1 = p0 * x;
    const double p2 = p1 * x;
    const double c0 = p0;
    const double c1 = c0 + p1;
    const double c2 = c1 + p2;
    theta[0] = cut_point(c0);
    theta[1] = cut_point(c1);
    theta[2] = cut_point(c2);
    return MICSA_OK;
}

int micsa_metro_thresholds(double T, uint64_t theta[3]) {
    if (!theta || !temperature_ok(T)) return MICSA_E_INVALID_ARG;
    const double beta = 1.0 / T;
    for (int k = 0; k < 3; ++k) theta[k] = cut_point(std::exp(-beta * 4.0 * (k + 1)));
    return MICSA_OK;
}

const char *micsa_last_error(micsa_t h) {
    if (!h) return "invalid handle (NULL)";
    return h->err.c_str();
}

void micsa_destroy(micsa_t h) {
    if (!h) return;
    DeviceGuard dg(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    cudaFree(h->d_spins);
    cudaFree(h->d_daemons);
    cudaFree(h->d_bonds);
    cudaFree(h->d_meas);
    cudaFree(h->d_stage);
    cudaFree(h->d_first);
    cudaFree(h->d_cursor);
    cudaFree(h->d_units);
    cudaFree(h->d_planes);
    cudaFree(h->d_bplanes);
    cudaFree(h->d_oc_nbrs);
    cudaFree(h->d_oc_flags);
    cudaFree(h->d_error);
    for (int c = 0; c < 3; ++c) {
        if (h->aux_stream[c]) cudaStreamDestroy(h->aux_stream[c]);
        if (h->join_ev[c]) cudaEventDestroy(h->join_ev[c]);
    }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    cudaFree(h->d_params);
    cudaFreeHost(h->h_params);
    drop_graphs(h);
    if (h->params_free) cudaEventDestroy(h->params_free);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
}

int micsa_create(int L, int n_samples, int n_replicas, uint64_t seed, micsa_t *out) {
    return micsa_create_ex(L, n_samples, n_replicas, 1, 0, seed, out);
}

int micsa_create_ex(int L, int n_samples, int n_replicas, int gamma, int walkers, uint64_t seed, micsa_t *out) {
    if (!out) return MICSA_E_INVALID_ARG;
    *out = nullptr;
    if (L < 2 || L > 1600 || (L & 1) || n_samples < 1 || n_replicas < 1 || n_replicas > 128 || gamma < 1 ||
        gamma > 8 || (int64_t)n_samples * n_replicas * gamma >= (1ll << 30))
        return MICSA_E_INVALID_ARG;
    micsa_ctx *h = new (std::nothrow) micsa_ctx;
    if (!h) return MICSA_E_OOM;
    h->L = L;
    h->S = n_samples;
    h->R = n_replicas;
    h->gamma = gamma;
    h->walkers = walkers ? 1 : 0;
    h->seed = seed;
    h->geo = make_geometry(L);
    int rc = MICSA_OK;
    do {
        if (cudaGetDevice(&h->device) != cudaSuccess) { rc = cuda_fail(h, cudaGetLastError(), "cudaGetDevice"); break; }
        cudaError_t e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { rc = cuda_fail(h, e, "cudaStreamCreate"); break; }
        h->stream = h->own_stream;
        if ((e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking)) != cudaSuccess) { rc = cuda_fail(h, e, "cudaStreamCreate"); break; }
        if ((e = cudaEventCreateWithFlags(&h->params_free, cudaEventDisableTiming)) != cudaSuccess) { rc = cuda_fail(h, e, "cudaEventCreate"); break; }
        if ((e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess) { rc = cuda_fail(h, e, "SM count"); break; }
        if ((e = cudaMalloc(&h->d_cursor, sizeof(int64_t))) != cudaSuccess) { rc = cuda_fail(h, e, "cudaMalloc cursor"); break; }
        const size_t state = (size_t)h->S * h->R * 2 * h->geo.half;
        const size_t dstate = state * (size_t)h->gamma;
        const size_t bonds = (size_t)h->S * 2 * h->geo.half;
        const size_t meas = sizeof(unsigned long long) * ((size_t)2 * h->S * h->R + (size_t)h->S * h->R * (h->R - 1) / 2);
        if ((e = cudaMalloc(&h->d_spins, state)) != cudaSuccess) { rc = cuda_fail(h, e, "cudaMalloc spins"); break; }
        if ((e = cudaMalloc(&h->d_daemons, dstate)) != cudaSuccess) { rc = cuda_fail(h, e, "cudaMalloc daemons"); break; }
        if ((e = cudaMalloc(&h->d_bonds, bonds)) != cudaSuccess) { rc = cuda_fail(h, e, "cudaMalloc bonds"); break; }
        if ((e = cudaMalloc(&h->d_meas, meas)) != cudaSuccess) { rc = cuda_fail(h, e, "cudaMalloc measure"); break; }
        if (resident_smem_bytes(h->geo) > 0) {
            std::vector<ResidentUnit> units((size_t)h->S * h->R);
            for (int a = 0; a < h->S; ++a)
                for (int r = 0; r < h->R; ++r) {
                    const int64_t gid = (int64_t)a * h->R + r;
                    units[gid] = ResidentUnit{h->d_spins + gid * 2 * h->geo.half, h->d_daemons + gid * 2 * h->geo.half,
                                              h->d_bonds + (int64_t)a * 2 * h->geo.half, (int32_t)gid, -1};
                }
            if ((e = cudaMalloc(&h->d_units, sizeof(ResidentUnit) * units.size())) != cudaSuccess) { rc = cuda_fail(h, e, "cudaMalloc units"); break; }
            if ((e = cudaMemcpy(h->d_units, units.data(), sizeof(ResidentUnit) * units.size(), cudaMemcpyHostToDevice)) != cudaSuccess) { rc = cuda_fail(h, e, "upload units"); break; }
        }
        h->device_bytes = state + dstate + bonds + meas;
        if ((e = cudaMemsetAsync(h->d_spins, 0, state, h->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(h->d_daemons, 0, dstate, h->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(h->d_bonds, 0, bonds, h->stream)) != cudaSuccess) { rc = cuda_fail(h, e, "cudaMemset"); break; }
        if ((rc = init_from_seed(h, seed)) != MICSA_OK) break;
        if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) { rc = cuda_fail(h, e, "create synchronize"); break; }
    } while (0);
    if (rc != MICSA_OK) {
        micsa_destroy(h);
        return rc;
    }
    *out = h;
    return MICSA_OK;
}

int micsa_reinit(micsa_t h, uint64_t seed) {
    if (!h) return MICSA_E_INVALID_ARG;
    DeviceGuard dg(h->device);
    return init_from_seed(h, seed);
}

int micsa_set_couplings(micsa_t h, const int8_t *J) {
    if (!h) return MICSA_E_INVALID_ARG;
    if (!J) return fail(h, MICSA_E_INVALID_ARG, "J is NULL");
    const int64_t n = sites(h) * 3 * h->S;
    DeviceGuard dg(h->device);
    if (int rc = ensure_stage(h, (size_t)n)) return rc;
    CK(h, cudaMemcpyAsync(h->d_stage, J, (size_t)n, cudaMemcpyHostToDevice, h->stream), "copy J");
    int64_t bad = -1;
    if (int rc = staged_first_invalid(h, h->d_stage, n, 0, &bad)) return rc;
    if (bad >= 0) return fail(h, MICSA_E_INVALID_ARG, "J[%lld] = %d is not +-1", (long long)bad, J[bad]);
    CK(h, launch_pack_couplings(h->d_bonds, reinterpret_cast<const int8_t *>(h->d_stage), h->geo, h->S, h->stream), "pack couplings");
    ++h->launches;
    CK(h, cudaStreamSynchronize(h->stream), "set_couplings synchronize");
    return MICSA_OK;
}

int micsa_get_couplings(micsa_t h, int8_t *J) {
    if (!h) return MICSA_E_INVALID_ARG;
    if (!J) return fail(h, MICSA_E_INVALID_ARG, "J is NULL");
    const int64_t n = sites(h) * 3 * h->S;
    DeviceGuard dg(h->device);
    if (int rc = ensure_stage(h, (size_t)n)) return rc;
    CK(h, launch_unpack_couplings(reinterpret_cast<int8_t *>(h->d_stage), h->d_bonds, h->geo, h->S, h->stream), "unpack couplings");
    ++h->launches;
    CK(h, cudaMemcpyAsync(J, h->d_stage, (size_t)n, cudaMemcpyDeviceToHost, h->stream), "copy J");
    CK(h, cudaStreamSynchronize(h->stream), "get_couplings synchronize");
    return MICSA_OK;
}

int micsa_run(micsa_t h, const double *schedule, int64_t n_sweeps, int32_t refresh_interval) {
    if (!h) return MICSA_E_INVALID_ARG;
    if (refresh_interval < 1) return fail(h, MICSA_E_INVALID_ARG, "refresh_interval must be >= 1");
    return run_micsa(h, schedule, n_sweeps, [=](int64_t t) { return t % refresh_interval == 0; });
}

int micsa_run_logrefresh(micsa_t h, const double *schedule, int64_t n_sweeps) {
    return run_micsa(h, schedule, n_sweeps, [](int64_t t) {
        const uint64_t v = (uint64_t)t + 1;
        return (v & (v - 1)) == 0;
    });
}

int micsa_run_metropolis(micsa_t h, const double *schedule, int64_t n_sweeps) {
    if (!h) return MICSA_E_INVALID_ARG;
    if (!schedule_ok(h, schedule, n_sweeps)) return MICSA_E_INVALID_ARG;
    if (n_sweeps == 0) return MICSA_OK;
    DeviceGuard dg(h->device);
    if (int rc = ensure_params(h, n_sweeps)) return rc;
    double last_T = -1.0;
    uint64_t th[3] = {0, 0, 0};
    for (int64_t k = 0; k < n_sweeps; ++k) {
        SweepParam &q = h->h_params[k];
        q.t = h->t + k;
        q.mode = kModeMetro;
        q.alpha = 0;
        if (schedule[k] != last_T) {
            micsa_metro_thresholds(schedule[k], th);
            last_T = schedule[k];
        }
        q.th0 = th[0];
        q.th1 = th[1];
        q.th2 = th[2];
    }
    if (int rc = run_table(h, true, n_sweeps)) return rc;
    h->t += n_sweeps;
    return MICSA_OK;
}

int micsa_set_launch_config(micsa_t h, int words_per_thread, int block, int blocks_per_sm, int pdl,
                            int graph_sweeps) {
    if (!h) return MICSA_E_INVALID_ARG;
    const bool regcap = (words_per_thread & MICSA_LAUNCH_REGCAP) != 0;
    const bool pairs = (words_per_thread & MICSA_LAUNCH_PAIRS) != 0;
    const bool reps = (words_per_thread & MICSA_LAUNCH_REPS) != 0;
    words_per_thread &= ~(MICSA_LAUNCH_REGCAP | MICSA_LAUNCH_PAIRS | MICSA_LAUNCH_REPS);
    if ((words_per_thread != 1 && words_per_thread != 2 && words_per_thread != 4) ||
        block < 32 || block > 256 || block % 32 || blocks_per_sm < -1 || blocks_per_sm > 64 ||
        graph_sweeps < 0 || graph_sweeps > 4096)
        return fail(h, MICSA_E_INVALID_ARG, "bad launch configuration");
    DeviceGuard dg(h->device);
    CK(h, cudaStreamSynchronize(h->stream), "synchronize before reconfiguring");
    drop_graphs(h);
    h->lc.nw = words_per_thread;
    h->lc.regcap = regcap;
    h->lc.pairs = pairs;
    h->lc.reps = reps && !pairs;
    h->lc.block = block;
    h->lc.pdl = pdl != 0;
    h->lc.graph_sweeps = graph_sweeps;
    h->blocks_per_sm = blocks_per_sm;
    return MICSA_OK;
}

int micsa_set_engine(micsa_t h, int engine, int resident_sweeps) {
    if (!h) return MICSA_E_INVALID_ARG;
    if (engine < MICSA_ENGINE_AUTO || engine > MICSA_ENGINE_TMA || resident_sweeps < 1 ||
        resident_sweeps > 1 << 20)
        return fail(h, MICSA_E_INVALID_ARG, "bad engine selection");
    if (engine == MICSA_ENGINE_MULTISPIN_GLOBAL && !msg_supported(h->geo))
        return fail(h, MICSA_E_INVALID_ARG, "the global multispin engine needs L a multiple of 32 (L=%d)", h->L);
    if (engine == MICSA_ENGINE_RESIDENT && resident_smem_bytes(h->geo) == 0)
        return fail(h, MICSA_E_INVALID_ARG, "an L=%d replica does not fit in shared memory", h->L);
    if (engine == MICSA_ENGINE_MULTISPIN && multispin_smem_bytes(h->geo) == 0)
        return fail(h, MICSA_E_INVALID_ARG, "the multispin engine needs L <= 32 (L=%d)", h->L);
    DeviceGuard dg(h->device);
    CK(h, cudaStreamSynchronize(h->stream), "synchronize before reconfiguring");
    if (engine == MICSA_ENGINE_ONCHIP)
        if (int rc = plan_onchip(h, effective_config(h, false).nw)) return rc;
    if (engine == MICSA_ENGINE_TMA)
        if (int rc = plan_tma(h)) return rc;
    drop_graphs(h);  // captured graphs hold the previous engine's kernels
    h->engine = engine;
    h->resident_sweeps = resident_sweeps;
    return MICSA_OK;
}

int micsa_set_replica_chains(micsa_t h, int chains) {
    if (!h) return MICSA_E_INVALID_ARG;
    if (chains < 1 || chains > 4) return fail(h, MICSA_E_INVALID_ARG, "replica chains must be in 1..4");
    DeviceGuard dg(h->device);
    CK(h, cudaStreamSynchronize(h->stream), "synchronize before reconfiguring");
    drop_graphs(h);
    h->chains = chains;
    return MICSA_OK;
}

int micsa_set_multispin_replicas(micsa_t h, int replicas_per_thread) {
    if (!h) return MICSA_E_INVALID_ARG;
    if (replicas_per_thread < 0 || replicas_per_thread > h->R)
        return fail(h, MICSA_E_INVALID_ARG, "replicas per thread must be in 0..%d", h->R);
    DeviceGuard dg(h->device);
    CK(h, cudaStreamSynchronize(h->stream), "synchronize before reconfiguring");
    drop_graphs(h);
    h->msg_rpt = replicas_per_thread;
    return MICSA_OK;
}

int micsa_get_engine(micsa_t h, int *engine) {
    if (!h || !engine) return MICSA_E_INVALID_ARG;
    *engine = active_engine(h);
    return MICSA_OK;
}

int micsa_get_launch_config(micsa_t h, int *words_per_thread, int *block, int *blocks_per_sm,
                            int *pdl, int *graph_sweeps) {
    if (!h) return MICSA_E_INVALID_ARG;
    const LaunchConfig lc = effective_config(h, false);
    if (words_per_thread)
        *words_per_thread = lc.nw | (lc.regcap ? MICSA_LAUNCH_REGCAP : 0) | (lc.pairs ? MICSA_LAUNCH_PAIRS : 0) |
                            (lc.reps ? MICSA_LAUNCH_REPS : 0);
    if (block) *block = lc.block;
    if (blocks_per_sm) *blocks_per_sm = h->blocks_per_sm;
    if (pdl) *pdl = lc.pdl;
    if (graph_sweeps) *graph_sweeps = lc.graph_sweeps;
    return MICSA_OK;
}

int micsa_measure(micsa_t h, int64_t *energy, int64_t *aux, int64_t *overlap) {
    if (!h) return MICSA_E_INVALID_ARG;
    DeviceGuard dg(h->device);
    if (int rc = check_device_error(h)) return rc;
    const size_t SR = (size_t)h->S * h->R;
    const size_t npair = (size_t)h->S * h->R * (h->R - 1) / 2;
    const size_t n = 2 * SR + npair;
    CK(h, cudaMemsetAsync(h->d_meas, 0, n * sizeof(unsigned long long), h->stream), "memset measure");
    CK(h, launch_measure(h->d_spins, h->d_daemons, h->d_bonds, h->geo, h->S, h->R, h->gamma, h->d_meas, h->stream), "measure launch");
    ++h->launches;
    std::vector<long long> host(n);
    CK(h, cudaMemcpyAsync(host.data(), h->d_meas, n * sizeof(long long), cudaMemcpyDeviceToHost, h->stream), "copy measure");
    CK(h, cudaStreamSynchronize(h->stream), "measure synchronize");
    if (energy) std::memcpy(energy, host.data(), SR * sizeof(int64_t));
    if (aux) std::memcpy(aux, host.data() + SR, SR * sizeof(int64_t));
    if (overlap && npair) std::memcpy(overlap, host.data() + 2 * SR, npair * sizeof(int64_t));
    return MICSA_OK;
}

int micsa_correlation(micsa_t h, int64_t *G) {
    if (!h) return MICSA_E_INVALID_ARG;
    if (!G) return fail(h, MICSA_E_INVALID_ARG, "G is NULL");
    if (h->R < 2) return fail(h, MICSA_E_INVALID_ARG, "the correlation needs two replicas or more");
    if (h->L > 1024) return fail(h, MICSA_E_INVALID_ARG, "the correlation supports L <= 1024");
    DeviceGuard dg(h->device);
    const int64_t npair = (int64_t)h->R * (h->R - 1) / 2;
    const size_t qbytes = (size_t)(sites(h) * h->S * npair);
    if (qbytes > ((size_t)4 << 30))
        return fail(h, MICSA_E_TOO_LARGE, "the overlap fields need %zu bytes of scratch (limit 4 GiB)", qbytes);
    const size_t gbytes = sizeof(long long) * (size_t)h->S * h->L;
    // scratch: the overlap fields, then the sums (16-byte aligned)
    const size_t goff = (qbytes + 15) / 16 * 16;
    if (int rc = ensure_stage(h, goff + gbytes)) return rc;
    unsigned long long *dG = reinterpret_cast<unsigned long long *>(h->d_stage + goff);
    CK(h, cudaMemsetAsync(dG, 0, gbytes, h->stream), "clear correlation sums");
    CK(h, launch_correlation(h->d_spins, h->geo, h->S, h->R, reinterpret_cast<int8_t *>(h->d_stage), dG, h->stream),
       "correlation launch");
    h->launches += 2;
    CK(h, cudaMemcpyAsync(G, dG, gbytes, cudaMemcpyDeviceToHost, h->stream), "copy correlation");
    CK(h, cudaStreamSynchronize(h->stream), "correlation synchronize");
    return MICSA_OK;
}

int micsa_c4(micsa_t h, double *C4) {
    if (!h) return MICSA_E_INVALID_ARG;
    if (!C4) return fail(h, MICSA_E_INVALID_ARG, "C4 is NULL");
    std::vector<int64_t> G((size_t)h->S * h->L);
    if (int rc = micsa_correlation(h, G.data())) return rc;
    // each unordered replica pair once, the three axes averaged: C4(0) = 1
    const double norm = 3.0 * (double)sites(h) * ((double)h->R * (h->R - 1) / 2);
    for (size_t i = 0; i < G.size(); ++i) C4[i] = (double)G[i] / norm;
    return MICSA_OK;
}

int micsa_get_state(micsa_t h, int8_t *spins, uint8_t *daemons, int64_t *t) {
    if (!h) return MICSA_E_INVALID_ARG;
    DeviceGuard dg(h->device);
    if (int rc = check_device_error(h)) return rc;
    const int64_t n = (int64_t)h->S * h->R;
    const size_t bytes = (size_t)(n * sites(h));
    const size_t dbytes = bytes * (size_t)h->gamma;
    if (spins || daemons) {
        if (int rc = ensure_stage(h, dbytes)) return rc;
    }
    if (spins) {
        CK(h, launch_convert_sites(reinterpret_cast<uint8_t *>(h->d_spins), h->d_stage, h->geo, n, false, h->stream), "gather spins");
        ++h->launches;
        CK(h, cudaMemcpyAsync(spins, h->d_stage, bytes, cudaMemcpyDeviceToHost, h->stream), "copy spins");
        CK(h, cudaStreamSynchronize(h->stream), "get_state synchronize");
    }
    if (daemons) {
        CK(h, launch_convert_sites(h->d_daemons, h->d_stage, h->geo, n * h->gamma, false, h->stream), "gather daemons");
        ++h->launches;
        CK(h, cudaMemcpyAsync(daemons, h->d_stage, dbytes, cudaMemcpyDeviceToHost, h->stream), "copy daemons");
        CK(h, cudaStreamSynchronize(h->stream), "get_state synchronize");
    }
    if (t) *t = h->t;
    return MICSA_OK;
}

int micsa_set_state(micsa_t h, const int8_t *spins, const uint8_t *daemons, int64_t t) {
    if (!h) return MICSA_E_INVALID_ARG;
    if (t < 0) return fail(h, MICSA_E_INVALID_ARG, "t must be >= 0");
    const int64_t n = (int64_t)h->S * h->R;
    const size_t bytes = (size_t)(n * sites(h));
    const size_t dbytes = bytes * (size_t)h->gamma;
    DeviceGuard dg(h->device);
    const size_t total = (spins ? bytes : 0) + (daemons ? dbytes : 0);
    if (total) {
        if (int rc = ensure_stage(h, total)) return rc;
    }
    uint8_t *s_stage = h->d_stage, *m_stage = h->d_stage + (spins ? bytes : 0);
    // both arrays are copied and checked on the device before either is written
    int64_t bad = -1;
    if (spins) {
        CK(h, cudaMemcpyAsync(s_stage, spins, bytes, cudaMemcpyHostToDevice, h->stream), "copy spins");
        if (int rc = staged_first_invalid(h, s_stage, (int64_t)bytes, 0, &bad)) return rc;
        if (bad >= 0) return fail(h, MICSA_E_INVALID_ARG, "spins[%lld] = %d is not +-1", (long long)bad, spins[bad]);
    }
    if (daemons) {
        CK(h, cudaMemcpyAsync(m_stage, daemons, dbytes, cudaMemcpyHostToDevice, h->stream), "copy daemons");
        if (int rc = staged_first_invalid(h, m_stage, (int64_t)dbytes, 1, &bad)) return rc;
        if (bad >= 0) return fail(h, MICSA_E_INVALID_ARG, "daemons[%lld] = %u exceeds 3", (long long)bad, daemons[bad]);
    }
    if (spins) {
        CK(h, launch_convert_sites(reinterpret_cast<uint8_t *>(h->d_spins), s_stage, h->geo, n, true, h->stream), "scatter spins");
        ++h->launches;
    }
    if (daemons) {
        CK(h, launch_convert_sites(h->d_daemons, m_stage, h->geo, n * h->gamma, true, h->stream), "scatter daemons");
        ++h->launches;
    }
    if (total) CK(h, cudaStreamSynchronize(h->stream), "set_state synchronize");
    h->t = t;
    return MICSA_OK;
}

int micsa_set_stream(micsa_t h, void *stream) {
    if (!h) return MICSA_E_INVALID_ARG;
    DeviceGuard dg(h->device);
    CK(h, cudaStreamSynchronize(h->stream), "synchronize old stream");
    h->stream = stream ? reinterpret_cast<cudaStream_t>(stream) : h->own_stream;
    return MICSA_OK;
}

int micsa_sync(micsa_t h) {
    if (!h) return MICSA_E_INVALID_ARG;
    DeviceGuard dg(h->device);
    CK(h, cudaStreamSynchronize(h->stream), "synchronize");
    return check_device_error(h);
}

int micsa_wait_selftest(int64_t polls, int *timed_out) {
    if (!timed_out || polls < 0) return MICSA_E_INVALID_ARG;
    *timed_out = 0;
    unsigned *flag = nullptr;
    int *err = nullptr;
    int v = 0, rc = MICSA_OK;
    if (cudaMalloc(&flag, sizeof(unsigned)) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess ||
        cudaMemset(flag, 0, sizeof(unsigned)) != cudaSuccess || cudaMemset(err, 0, sizeof(int)) != cudaSuccess ||
        launch_wait_selftest(flag, err, (long long)polls, nullptr) != cudaSuccess ||
        cudaMemcpy(&v, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = MICSA_E_CUDA;
    cudaFree(flag);
    cudaFree(err);
    *timed_out = v;
    return rc;
}

int micsa_launch_count(micsa_t h, int64_t *count) {
    if (!h || !count) return MICSA_E_INVALID_ARG;
    *count = h->launches;
    return MICSA_OK;
}

int micsa_device_bytes(micsa_t h, size_t *bytes) {
    if (!h || !bytes) return MICSA_E_INVALID_ARG;
    *bytes = h->device_bytes;
    return MICSA_OK;
}

}  // extern "C"
