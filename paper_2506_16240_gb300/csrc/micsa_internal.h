// micsa_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "micsa_device.cuh"

namespace micsa {

enum { kModeMicsa = 0, kModeRefresh = 1, kModeMetro = 2 };

struct SweepArgs {
    int8_t *spins;        // [S][R][2][half]
    uint8_t *daemons;     // [S][R][2][half]
    const uint8_t *bonds; // [S][2][half]
    Geometry geo;
    int S, R;
    int parity;
    uint32_t key0, key1;  // Philox key = seed
    int64_t t;            // global sweep index of this half-sweep
    uint64_t th0, th1, th2;  // refresh (daemon) or Metropolis cut points
};

// word loads/stores of NW consecutive 32-bit words; NW == 4 uses one 16-byte
// access (the caller guarantees 16-byte alignment in that case)
template <int NW>
__device__ __forceinline__ void load_words(const void *p, uint32_t (&w)[NW]) {
    if constexpr (NW == 4) {
        const uint4 v = *reinterpret_cast<const uint4 *>(p);
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
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
    } else {
#pragma unroll
        for (int j = 0; j < NW; ++j) w[j] = __ldg(reinterpret_cast<const uint32_t *>(p) + j);
    }
}

template <int NW>
__device__ __forceinline__ void store_words(void *p, const uint32_t (&w)[NW]) {
    if constexpr (NW == 4) {
        *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    } else {
#pragma unroll
        for (int j = 0; j < NW; ++j) reinterpret_cast<uint32_t *>(p)[j] = w[j];
    }
}

Geometry make_geometry(int L);

cudaError_t launch_half_sweep(const SweepArgs &a, int mode, cudaStream_t st);

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
