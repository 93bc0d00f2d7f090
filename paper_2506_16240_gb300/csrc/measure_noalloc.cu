// measure_noalloc.cu -- observables of caller-owned device arrays with no
// device allocation at all.
//
// Who needs this: code that must not call cudaMalloc -- a host framework whose
// caching allocator owns all device memory and must account for every byte, a
// serving loop that cannot afford the implicit device synchronisation an
// allocation may cause, or a process running under a fixed memory budget. Such
// callers hold the spins, daemons and couplings in their own device buffers and
// only want the exact energies and overlaps back.
//
// The per-call accumulators live in one file-scope device array of fixed size
// (kMaxTerms 64-bit counters, 64 KiB) that every GPU loading this library keeps
// until the process exits. Host code cannot use the array's name as a device
// address, so its address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernel. The array is shared by all
// calls: each call clears the part it uses first, and calls whose GPU work
// overlaps (different streams, or host threads) race on it.
#include <cstdio>
#include <mutex>

#include "micsa_internal.h"
#include "../../include/micsa.h"

namespace {

constexpr int kMaxTerms = MICSA_NOALLOC_MAX_TERMS;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned long long g_noalloc_scratch[kMaxTerms];

unsigned long long *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Device address of the scratch array on the current device, looked up on the
// first call per device (that call must come before any stream capture) and
// kept for the life of the process (stale after cudaDeviceReset).
cudaError_t scratch_address(unsigned long long **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// One thread per site of one sample (blockIdx.y). Energy over the three forward
// bonds of each site, Eq. (Hamiltonian); H_aux = 4 sum m; overlaps of replica
// pairs. Block sums in shared memory, then one atomic per block and term into
// `acc` = [energy S*R | aux S*R | overlap S*R(R-1)/2].
__global__ void __launch_bounds__(256) measure_natural_kernel(const int8_t *spins, const uint8_t *daemons,
                                                              const int8_t *J, int L, int S, int R,
                                                              unsigned long long *acc) {
    extern __shared__ long long part[];
    const int npair = R * (R - 1) / 2;
    const int nq = 2 * R + npair;
    for (int i = threadIdx.x; i < nq; i += blockDim.x) part[i] = 0;
    __syncthreads();

    const int sample = blockIdx.y;
    const int64_t N = (int64_t)L * L * L;
    const int64_t site = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = site < N;
    int x = 0, y = 0, z = 0;
    if (active) {
        x = (int)(site % L);
        y = (int)((site / L) % L);
        z = (int)(site / ((int64_t)L * L));
    }
    const int64_t nb[3] = {((int64_t)z * L + y) * L + (x + 1 == L ? 0 : x + 1),
                           ((int64_t)z * L + (y + 1 == L ? 0 : y + 1)) * L + x,
                           ((int64_t)(z + 1 == L ? 0 : z + 1) * L + y) * L + x};
    const int8_t *Js = J + ((int64_t)sample * N + site) * 3;
    const int lane = threadIdx.x & 31;

    for (int r = 0; r < R; ++r) {
        const int8_t *s = spins + ((int64_t)sample * R + r) * N;
        int e = 0, a = 0;
        if (active) {
            const int sx = s[site];
            for (int d = 0; d < 3; ++d) e -= Js[d] * sx * s[nb[d]];
            if (daemons) a = 4 * daemons[((int64_t)sample * R + r) * N + site];
        }
        e = __reduce_add_sync(0xFFFFFFFFu, e);
        a = __reduce_add_sync(0xFFFFFFFFu, a);
        if (lane == 0) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&part[r]), (unsigned long long)(long long)e);
            atomicAdd(reinterpret_cast<unsigned long long *>(&part[R + r]), (unsigned long long)(long long)a);
        }
    }
    int pair = 0;
    for (int ra = 0; ra < R; ++ra)
        for (int rb = ra + 1; rb < R; ++rb, ++pair) {
            int q = 0;
            if (active)
                q = spins[((int64_t)sample * R + ra) * N + site] * spins[((int64_t)sample * R + rb) * N + site];
            q = __reduce_add_sync(0xFFFFFFFFu, q);
            if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long *>(&part[2 * R + pair]), (unsigned long long)(long long)q);
        }
    __syncthreads();
    for (int i = threadIdx.x; i < nq; i += blockDim.x) {
        const long long v = part[i];
        if (v == 0) continue;
        int64_t dst;
        if (i < R) dst = (int64_t)sample * R + i;
        else if (i < 2 * R) dst = (int64_t)S * R + (int64_t)sample * R + (i - R);
        else dst = 2 * (int64_t)S * R + (int64_t)sample * npair + (i - 2 * R);
        atomicAdd(acc + dst, (unsigned long long)v);
    }
}

}  // namespace

extern "C" int micsa_measure_noalloc(const int8_t *spins, const uint8_t *daemons, const int8_t *J, int L,
                                     int n_samples, int n_replicas, int64_t *energy, int64_t *aux,
                                     int64_t *overlap, void *stream) {
    if (!spins || !J || L < 2 || L > 1600 || n_samples < 1 || n_replicas < 1 || n_replicas > 32)
        return MICSA_E_INVALID_ARG;
    const int64_t SR = (int64_t)n_samples * n_replicas;
    const int64_t npair = (int64_t)n_samples * n_replicas * (n_replicas - 1) / 2;
    const int64_t terms = 2 * SR + npair;
    if (terms > kMaxTerms || n_samples > 65535) return MICSA_E_TOO_LARGE;
    unsigned long long *acc = nullptr;
    cudaError_t e = scratch_address(&acc);
    if (e != cudaSuccess) return MICSA_E_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the array keeps the previous call's sums: clear what this call uses
    if ((e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * (size_t)terms, st)) != cudaSuccess)
        return MICSA_E_CUDA;
    const int64_t N = (int64_t)L * L * L;
    const dim3 grid((unsigned)((N + 255) / 256), (unsigned)n_samples);
    const int nq = 2 * n_replicas + n_replicas * (n_replicas - 1) / 2;
    measure_natural_kernel<<<grid, 256, sizeof(long long) * nq, st>>>(spins, daemons, J, L, n_samples,
                                                                      n_replicas, acc);
    if ((e = cudaGetLastError()) != cudaSuccess) return MICSA_E_CUDA;
    // copy the three parts of the sums straight into the caller's host arrays
    if (energy && (e = cudaMemcpyAsync(energy, acc, sizeof(int64_t) * SR, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return MICSA_E_CUDA;
    if (aux && (e = cudaMemcpyAsync(aux, acc + SR, sizeof(int64_t) * SR, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return MICSA_E_CUDA;
    if (overlap && npair &&
        (e = cudaMemcpyAsync(overlap, acc + 2 * SR, sizeof(int64_t) * npair, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return MICSA_E_CUDA;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return MICSA_E_CUDA;
    return MICSA_OK;
}
