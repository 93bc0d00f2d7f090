// micsa_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "micsa_device.cuh"

namespace micsa {

enum { kModeMicsa = 0, kModeRefresh = 1, kModeMetro = 2 };

// Parameters of one sweep of a run, uploaded as a table before the run.
struct SweepParam {
    int64_t t;               // global sweep index (Philox counter word)
    uint64_t th0, th1, th2;  // refresh (daemon) or Metropolis cut points
    int32_t mode;            // kModeMicsa or kModeRefresh; unused by Metropolis
    int32_t pad;
};

struct SweepArgs {
    int8_t *spins;        // [S][R][2][half]
    uint8_t *daemons;     // [S][R][2][half]
    const uint8_t *bonds; // [S][2][half]
    Geometry geo;
    int S, R;
    int parity;
    uint32_t key0, key1;         // Philox key = seed
    const SweepParam *params;    // the run's table
    const int64_t *cursor;       // graph replays: base index into params; else nullptr
    int64_t k;                   // this sweep's index relative to *cursor (or absolute)
};

// Launch shape of the half-sweep kernels (picked by the autotuner; results are
// identical for every choice).
struct LaunchConfig {
    int nw = 4;          // 32-bit words per thread (4, 2 or 1; reduced to what the pitch allows)
    int block = 128;     // threads per block (chunks x replica rows)
    int max_blocks = 0;  // grid cap for the grid-stride loop (0: one thread per chunk)
    bool pdl = true;     // programmatic dependent launch between consecutive grids
    int graph_sweeps = 64;  // sweeps per captured CUDA graph (0: no graphs)
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
cudaError_t launch_advance_cursor(int64_t *cursor, int64_t step, bool pdl, cudaStream_t st);
int vector_words(const Geometry &g, int want);
int max_resident_blocks(bool metro, int nw, int block);
dim3 block_shape(int R, int block);

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
cudaError_t launch_convert_sites(uint8_t *split, uint8_t *natural, Geometry g, int64_t n,
                                 bool to_split, cudaStream_t st);
cudaError_t launch_measure(const int8_t *spins, const uint8_t *daemons, const uint8_t *bonds,
                           Geometry g, int S, int R, unsigned long long *out, cudaStream_t st);

}  // namespace micsa
