// resident.cu -- the shared-memory resident kernel: a CTA copies a whole
// lattice replica (spins, daemons and bonds of both parities, 3 bytes per site)
// into shared memory, runs a block of K MicSA sweeps on it there -- even
// half-sweep, barrier, odd half-sweep, barrier, as in the procedure of
// Sec. 2.8 -- and copies spins and daemons back. Inside the block of sweeps no
// lattice byte touches L2 or HBM. The arithmetic is the update of
// sweep_body.cuh on shared-memory operands, so results are bit-identical to
// the streaming kernel.
//
// Two clocks:
//   handle mode: all units run sweeps k0 .. k0+K-1 of the run's parameter
//     table (any refresh pattern, Sec. 2.7 / 2.8);
//   pool mode: each unit belongs to a pool job with its own clock t, refresh
//     interval and cut-point table; after its sweeps the CTA measures the
//     exact energy and keeps the lowest one and its configuration.
#include "sweep_body.cuh"
#include "../../include/micsa.h"

namespace micsa {

constexpr int kResidentThreads = 512;
constexpr int kPoolMaxRes = MICSA_POOL_MAX_REPLICAS;

size_t resident_smem_bytes(const Geometry &g) {
    const size_t bytes = 6 * (size_t)g.half;  // spins, daemons, bonds; two parities each
    return bytes <= 200 * 1024 ? bytes : 0;
}

__device__ __forceinline__ void copy16(void *dst, const void *src, int64_t bytes) {
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    for (int64_t i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = s[i];
}

template <int NW>
__device__ __forceinline__ void resident_half(const Geometry &g, int8_t *sp, uint8_t *dm, const uint8_t *bd,
                                              int p, uint32_t gid, uint32_t k0, uint32_t k1, int64_t t,
                                              bool refresh, uint64_t th0, uint64_t th1, uint64_t th2) {
    const int chunks = g.W / NW;
    const int items = g.L * g.L * chunks;
    const FastDiv divL = make_fastdiv_dev((uint32_t)g.L);
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int row = it / chunks;
        const int c = it - row * chunks;
        update_chunk<NW, false, true>(g, sp, dm, bd, p, row, c, gid, k0, k1, t, refresh, th0, th1, th2, divL);
    }
}

__device__ __forceinline__ void grid_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <bool POOL>
__global__ void __launch_bounds__(kResidentThreads, 2) resident_kernel(ResidentArgs A) {
    grid_wait();
    grid_release();
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_unit;
    __shared__ long long s_red[2][kResidentThreads / 32];
    __shared__ int s_improved;

    const int n_units = A.n_units_dev ? *A.n_units_dev : A.n_units;
    for (int n_done = 0;; ++n_done) {
        int u;
        if (POOL) {
            if (threadIdx.x == 0) s_unit = atomicAdd(A.counter, 1);
            __syncthreads();
            u = s_unit;
        } else {
            u = blockIdx.x + n_done * gridDim.x;
        }
        if (u >= n_units) break;
        const ResidentUnit U = A.units[u];
        Geometry g = A.geo;
        uint32_t key0 = A.key0, key1 = A.key1;
        int64_t t0 = 0, n_sweeps = 0;
        int32_t interval = 1;
        const uint64_t *thr = nullptr;
        if (POOL) {
            const JobDesc &J = A.jobs[U.slot];
            g = J.geo;
            key0 = J.key0;
            key1 = J.key1;
            t0 = J.t;
            n_sweeps = J.n_sweeps;
            interval = J.interval;
            thr = J.thr;
            if (t0 >= n_sweeps) {  // finished: nothing to run or measure
                __syncthreads();
                continue;
            }
        }
        int8_t *sp = reinterpret_cast<int8_t *>(smem);
        uint8_t *dm = smem + 2 * g.half;
        uint8_t *bd = smem + 4 * g.half;
        copy16(sp, U.spins, 2 * g.half);
        copy16(dm, U.daemons, 2 * g.half);
        copy16(bd, U.bonds, 2 * g.half);
        __syncthreads();

        int64_t t_end = 0;
        for (int k = 0; k < A.K; ++k) {
            int64_t t;
            bool refresh;
            uint64_t th0 = 0, th1 = 0, th2 = 0;
            if (POOL) {
                t = t0 + k;
                if (t >= n_sweeps) break;
                refresh = (t % interval) == 0;
                if (refresh) {
                    const uint64_t *q = thr + 3 * (t / interval);
                    th0 = q[0];
                    th1 = q[1];
                    th2 = q[2];
                }
            } else {
                const SweepParam prm = A.params[A.k0 + k];
                t = prm.t;
                refresh = prm.mode == kModeRefresh;
                th0 = prm.th0;
                th1 = prm.th1;
                th2 = prm.th2;
            }
            for (int p = 0; p < 2; ++p) {
                if (g.W % 4 == 0)
                    resident_half<4>(g, sp, dm, bd, p, (uint32_t)U.gid, key0, key1, t, refresh, th0, th1, th2);
                else
                    resident_half<1>(g, sp, dm, bd, p, (uint32_t)U.gid, key0, key1, t, refresh, th0, th1, th2);
                __syncthreads();
            }
            t_end = t + 1;
        }
        copy16(U.spins, sp, 2 * g.half);
        copy16(U.daemons, dm, 2 * g.half);

        if (POOL) {
            // exact energy and daemon energy of the state just reached
            const int64_t words = (int64_t)g.L * g.L * g.W;
            long long e = 0, a = 0;
            for (int64_t w = threadIdx.x; w < words; w += blockDim.x) {
                e += even_word_energy<true>(g, sp, sp + g.half, bd, w);
                const int b0 = (int)(w % g.W) * 4;
                const uint32_t valid = valid_mask(b0, 0, g.Lh);
                const uint32_t D0 = *reinterpret_cast<const uint32_t *>(dm + 4 * w) & valid;
                const uint32_t D1 = *reinterpret_cast<const uint32_t *>(dm + g.half + 4 * w) & valid;
                a += 4 * (long long)(((D0 * 0x01010101u) >> 24) + ((D1 * 0x01010101u) >> 24));
            }
            e = __reduce_add_sync(0xFFFFFFFFu, (int)e);
            a = __reduce_add_sync(0xFFFFFFFFu, (int)a);
            if ((threadIdx.x & 31) == 0) {
                s_red[0][threadIdx.x >> 5] = e;
                s_red[1][threadIdx.x >> 5] = a;
            }
            __syncthreads();
            const int cell = U.slot * kPoolMaxRes + U.gid;
            const int64_t rows = (int64_t)A.max_jobs * kPoolMaxRes;
            if (threadIdx.x == 0) {
                long long es = 0, as = 0;
                for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
                    es += s_red[0][i];
                    as += s_red[1][i];
                }
                A.results[cell] = es;
                A.results[rows + cell] = as;
                s_improved = es < A.results[2 * rows + cell];
                if (s_improved) {
                    A.results[2 * rows + cell] = es;
                    A.results[3 * rows + cell] = t_end;
                }
            }
            __syncthreads();
            if (s_improved) {
                const JobDesc &J = A.jobs[U.slot];
                const int64_t N = (int64_t)g.L * g.L * g.L;
                int8_t *best = J.best + (int64_t)U.gid * N;
                for (int64_t site = threadIdx.x; site < N; site += blockDim.x) {
                    const int x = (int)(site % g.L), y = (int)((site / g.L) % g.L), z = (int)(site / ((int64_t)g.L * g.L));
                    const int par = (x + y + z) & 1;
                    best[site] = sp[(int64_t)par * g.half + ((int64_t)z * g.L + y) * g.P + (x >> 1)];
                }
            }
        }
        __syncthreads();  // shared memory is reused by the next unit
    }
}

cudaError_t launch_resident(const ResidentArgs &a, bool pool, size_t smem, int grid, bool pdl, cudaStream_t st) {
    const void *fn = pool ? (const void *)resident_kernel<true> : (const void *)resident_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kResidentThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ResidentArgs args = a;
    void *kargs[] = {&args};
    return cudaLaunchKernelExC(&cfg, fn, kargs);
}

int resident_blocks_per_sm(bool pool, size_t smem) {
    const void *fn = pool ? (const void *)resident_kernel<true> : (const void *)resident_kernel<false>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kResidentThreads, smem) != cudaSuccess) return 0;
    return n;
}

}  // namespace micsa
