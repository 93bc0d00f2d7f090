// micsa_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "micsa_device.cuh"

namespace micsa {

enum { kModeMicsa = 0, kModeRefresh = 1, kModeMetro = 2 };

// Parameters of one sweep of a run, uploaded as a table before the run.
struct SweepParam {
    int64_t t;               // global sweep index (Philox counter word)
    uint64_t th0, th1, th2;  // refresh (daemon) or Metropolis cut points
    int32_t mode;            // kModeMicsa or kModeRefresh; unused by Metropolis
    int32_t alpha;           // daemon family used by this sweep (0 .. gamma-1)
    int32_t gather;          // bit planes with walkers: the previous timestep's wandering step is
                             // applied on read (daemons gathered from the other buffer)
    int32_t reserved;
};

struct SweepArgs {
    int8_t *spins;        // [S][R][2][half]
    uint8_t *daemons;     // [S][R][2][half]
    const uint8_t *bonds; // [S][2][half]
    Geometry geo;
    int S, R;
    int gamma;                   // daemon families per spin (daemons: [S][R][gamma][2][half])
    int parity;
    uint32_t key0, key1;         // Philox key = seed
    const SweepParam *params;    // the run's table
    const int64_t *cursor;       // graph replays: base index into params; else nullptr
    int64_t k;                   // this sweep's index relative to *cursor (or absolute)
    int r0, r1;                  // replicas [r0, r1) of every sample are updated (0, R: all)
    FastDiv div_chunks;          // row pairs: divide by chunks per row as well
    FastDiv div_half_L;          // row pairs: divide by L / 2          // row -> (row, chunk): divide by chunks per row
    FastDiv div_L;               // row -> (z, y): divide by L
};

// Launch shape of the half-sweep kernels (picked by the autotuner; results are
// identical for every choice).
struct LaunchConfig {
    int nw = 4;          // 32-bit words per thread (4, 2 or 1; reduced to what the pitch allows)
    int block = 128;     // threads per block (chunks x replica rows)
    int max_blocks = 0;  // grid cap for the grid-stride loop (0: one thread per chunk)
    bool pdl = true;     // programmatic dependent launch between consecutive grids
    int graph_sweeps = 64;  // sweeps per captured CUDA graph (0: no graphs)
    bool regcap = false;    // kernel variant with registers capped at 64 (blocks of <= 128)
    int chains = 1;         // replica groups captured as concurrent kernel chains in one graph
    bool pairs = false;     // one thread updates two rows (rows without padding, MicSA only)
    bool reps = false;      // one thread updates its chunk for every replica (rows without padding, MicSA only)
};

// One job of the batched pool (device-resident descriptor).
struct JobDesc {
    int32_t resident;      // advanced by the shared-memory resident kernel
    int8_t *spins;         // [R][2][half]
    uint8_t *daemons;      // [R][2][half]
    const uint8_t *bonds;  // [2][half]
    int8_t *best;          // [R][N] natural layout
    const uint64_t *thr;   // refresh cut points [n_refresh][3]
    Geometry geo;
    int R, nw;
    uint32_t key0, key1;
    int64_t t;             // sweeps done
    int64_t n_sweeps;
    int32_t interval;
    int32_t live;
    uint32_t divL_m, divL_l;  // FastDiv by L
    uint32_t divC_m, divC_l;  // FastDiv by chunks per row (W / nw)
    // bit-plane jobs (L a multiple of 32): during a tick the state lives in
    // planes [R][6][L^3/64] (spins, m0, m1 of both parities), the bonds in
    // bplanes [6][2][L^3/64]; the byte arrays hold it between ticks
    uint32_t *planes;
    const uint32_t *bplanes;
    int32_t use_planes;
    int32_t smem_planes;  // bit-plane job swept in shared memory by the tick's persistent kernel: the
                          // per-CTA shared-memory budget (bytes) it was admitted with; 0: not
    int32_t smem_cluster;  // > 1: each of its shared-memory units is split over a cluster of this many CTAs
};

// One lattice (a replica of a sample or of a pool job) that a CTA keeps in
// shared memory while it runs a block of sweeps.
struct ResidentUnit {
    int8_t *spins;         // [2][half] of this replica
    uint8_t *daemons;      // [2][half]
    const uint8_t *bonds;  // [2][half] of its sample
    int32_t gid;           // replica id in the Philox counter
    int32_t slot;          // pool: job slot (clock, schedule, results); handle: -1
};

struct ResidentArgs {
    const ResidentUnit *units;
    int n_units;
    const int *n_units_dev;       // pool mode: unit count read on the device (graph replays)
    Geometry geo;                 // handle mode: the common geometry
    uint32_t key0, key1;          // handle mode: the common key
    const SweepParam *params;     // handle mode: sweep table
    int64_t k0;                   // handle mode: first sweep of this launch in the table
    int K;                        // sweeps per launch
    int *counter;                 // pool mode: work counter (reset by the tick's last node)
    const JobDesc *jobs;          // pool mode: job table
    long long *results;           // pool mode: energy | aux | best_energy | best_t rows
    int max_jobs;                 // pool mode: row length of each results array / kPoolMaxR
};

// word loads/stores of NW consecutive 32-bit words as one 4-, 8- or 16-byte
// access (the caller guarantees the matching alignment)
template <int NW>
__device__ __forceinline__ void load_words(const void *p, uint32_t (&w)[NW]) {
    if constexpr (NW == 4) {
        const uint4 v = *reinterpret_cast<const uint4 *>(p);
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else if constexpr (NW == 2) {
        const uint2 v = *reinterpret_cast<const uint2 *>(p);
        w[0] = v.x; w[1] = v.y;
    } else {
#pragma unroll
        for (int j = 0; j < NW; ++j) w[j] = reinterpret_cast<const uint32_t *>(p)[j];
    }
}

template <int NW>
__device__ __forceinline__ void load_words_ro(const void *p, uint32_t (&w)[NW]) {
    if constexpr (NW == 4) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else if constexpr (NW == 2) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        w[0] = v.x; w[1] = v.y;
    } else {
#pragma unroll
        for (int j = 0; j < NW; ++j) w[j] = __ldg(reinterpret_cast<const uint32_t *>(p) + j);
    }
}

template <int NW>
__device__ __forceinline__ void store_words(void *p, const uint32_t (&w)[NW]) {
    if constexpr (NW == 4) {
        *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    } else if constexpr (NW == 2) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(w[0], w[1]);
    } else {
#pragma unroll
        for (int j = 0; j < NW; ++j) reinterpret_cast<uint32_t *>(p)[j] = w[j];
    }
}

Geometry make_geometry(int L);

cudaError_t launch_half_sweep(const SweepArgs &a, bool metro, const LaunchConfig &lc, cudaStream_t st);

// shared-memory resident kernel (resident.cu)
size_t resident_smem_bytes(const Geometry &g);  // 0 when the lattice does not fit
cudaError_t launch_resident(const ResidentArgs &a, bool pool, size_t smem, int grid, bool pdl, cudaStream_t st);
int resident_blocks_per_sm(bool pool, size_t smem);

// multispin (bit-plane) resident kernel for L <= 32 (multispin.cu)
size_t multispin_smem_bytes(const Geometry &g);  // 0 when L > 32
cudaError_t launch_multispin(const ResidentArgs &a, bool pool, size_t smem, int grid, bool pdl, cudaStream_t st);
int multispin_blocks_per_sm(bool pool, size_t smem);

// persistent engine with the state in the shared memory of all SMs (onchip.cu)
struct OnchipPlan {
    int grid = 0, k = 0, qmax = 0, nw = 0;  // CTAs, CTAs per sample, rows per CTA, words per item
    size_t smem = 0;
    std::vector<int16_t> table;  // [grid][max neighbours], -1 terminated
};
bool onchip_plan(const Geometry &g, int S, int R, int ctas, int nw, OnchipPlan &plan);
size_t onchip_flag_words(int grid);
int onchip_max_neighbours();
cudaError_t launch_onchip(const OnchipPlan &plan, int8_t *spins, uint8_t *daemons, const uint8_t *bonds,
                          const Geometry &g, int S, int R, uint32_t key0, uint32_t key1, const SweepParam *params,
                          int64_t k0, int K, unsigned *flags, int *error, const int16_t *nbrs, long long wait_limit,
                          cudaStream_t st);
cudaError_t launch_wait_selftest(unsigned *flag, int *error, long long wait_limit, cudaStream_t st);

// half-sweep with TMA-staged tiles (tma_sweep.cu)
struct TmaMaps {
    CUtensorMap m_int, m_yh, m_zh, m_dmn, m_bond;  // spins (3 box shapes), daemons, bonds
    bool valid = false;
};
bool tma_supported(const Geometry &g, int gamma, int walkers);
cudaError_t tma_encode(TmaMaps &m, int8_t *spins, uint8_t *daemons, const uint8_t *bonds, const Geometry &g, int S,
                       int R);
int tma_stages(const Geometry &g);
int tma_max_ctas(const Geometry &g, int sm_count);
cudaError_t launch_tma_half(const TmaMaps &m, int8_t *spins, uint8_t *daemons, const Geometry &g, int S, int R,
                            int r0, int r1, int parity, uint32_t key0, uint32_t key1, const SweepParam *params,
                            const int64_t *cursor, int64_t k, int *error, long long wait_limit, int max_ctas,
                            bool pdl, cudaStream_t st);

// multispin planes in global memory for L % 32 == 0 (multispin.cu)
bool msg_supported(const Geometry &g);
int64_t msg_plane_words(const Geometry &g);  // words per parity plane, L * ceil(L / 32) * Lh
int msg_planes_per_replica(int gamma, int walkers);  // 2 spin + 4 gamma daemon planes (x 2 buffers)
cudaError_t msg_convert(uint32_t *planes, uint32_t *bplanes, int8_t *spins, uint8_t *daemons, const uint8_t *bonds,
                        const Geometry &g, int S, int R, int gamma, int walkers, int buf, bool to_planes,
                        cudaStream_t st);
cudaError_t msg_convert_bonds(uint32_t *bplanes, const uint8_t *bonds, const Geometry &g, int S, cudaStream_t st);
cudaError_t launch_msg_wander(uint32_t *planes, const Geometry &g, int S, int R, int r0, int r1, int gamma,
                              const SweepParam *params, const int64_t *cursor, int64_t k, bool pdl, cudaStream_t st);
int msg_default_rpt(const Geometry &g, int S, int R, int nw, int sm_count);
cudaError_t launch_msg_half(uint32_t *planes, const uint32_t *bplanes, const Geometry &g, int S, int R, int r0,
                            int r1, int rpt, int nw, bool regcap, int parity, int gamma, int walkers, uint32_t key0, uint32_t key1, const SweepParam *params,
                            const int64_t *cursor, int64_t k, bool pdl, cudaStream_t st, bool metro = false);
cudaError_t launch_advance_cursor(int64_t *cursor, int64_t step, bool pdl, cudaStream_t st);
// wandering of every walker family after timestep t (parity t & 1), Sec. 2.6
cudaError_t launch_wander(uint8_t *daemons, Geometry g, int64_t n_rep, int gamma, int parity, cudaStream_t st);
int vector_words(const Geometry &g, int want);
int max_resident_blocks(bool metro, int nw, int block, bool regcap);
int max_resident_blocks_pairs(int nw, int block);
int max_resident_blocks_reps(int nw, int block);
dim3 block_shape(int R, int block, int max_threads);

// initialisation, layout conversion and measurement (init_measure.cu)
cudaError_t launch_init_couplings(uint8_t *bonds, Geometry g, int S, uint32_t k0, uint32_t k1,
                                  cudaStream_t st);
cudaError_t launch_init_spins(int8_t *spins, Geometry g, int S, int R, uint32_t k0, uint32_t k1,
                              cudaStream_t st);
cudaError_t launch_pack_couplings(uint8_t *bonds, const int8_t *J_nat, Geometry g, int S,
                                  cudaStream_t st);
cudaError_t launch_unpack_couplings(int8_t *J_nat, const uint8_t *bonds, Geometry g, int S,
                                    cudaStream_t st);
// natural [n][N] <-> split [n][2][half]; `to_split` selects the direction
cudaError_t launch_first_invalid(const uint8_t *v, int64_t n, int mode, unsigned long long *first,
                                 cudaStream_t st);
cudaError_t launch_convert_sites(uint8_t *split, uint8_t *natural, Geometry g, int64_t n,
                                 bool to_split, cudaStream_t st);
cudaError_t launch_measure(const int8_t *spins, const uint8_t *daemons, const uint8_t *bonds,
                           Geometry g, int S, int R, int gamma, unsigned long long *out, cudaStream_t st);
// C4 sums G[S][L] (Sec. 3); q_scratch holds N * S * R(R-1)/2 bytes
cudaError_t launch_correlation(const int8_t *spins, Geometry g, int S, int R, int8_t *q_scratch,
                               unsigned long long *G, cudaStream_t st);

}  // namespace micsa
