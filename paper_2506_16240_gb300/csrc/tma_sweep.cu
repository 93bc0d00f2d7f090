// tma_sweep.cu -- the MicSA half-sweep on the byte layout with the tiles staged
// in shared memory by the Tensor Memory Accelerator (Sec. 2.8 steps (i), (ii);
// Eq. (Creutz) with Eq. (flip-OK); refresh of Sec. 2.7 fused in).
//
// The lattice halves are 4D tensors of bytes: x = the P bytes of a row, y, z,
// and n = the (replica, parity) half (bonds: the (sample, parity) half). A
// tile is 8 planes x 8 rows of full rows for a group of up to two replicas of
// one sample. Per tile and replica one TMA box brings the 8 x 8 rows of the
// opposite parity, two 8 x 1 boxes the rows y0 - 1 and y0 + 8, two 1 x 8
// boxes the planes z0 - 1 and z0 + 8 (coordinates taken mod L: the periodic
// halo), and 8 x 8 boxes the own spins and daemons (not on a refresh sweep);
// one box the bonds of the sample. A persistent CTA walks its tiles through a
// ring of 2..4 stages, one mbarrier each: the loads of the next tiles are in
// flight while a tile is updated from shared memory, and the updated spin and
// daemon words go back to global memory with 16-byte stores. Every mbarrier
// wait is bounded: on time-out the CTA records it in the error word, waits
// (bounded) for its loads still in flight and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "micsa_internal.h"

namespace micsa {

constexpr int kTmaT = 8;          // tile edge in rows (y) and planes (z)
constexpr int kTmaThreads = 512;
constexpr int kTmaRG = 2;         // replicas per tile
constexpr int kTmaMaxStages = 4;

struct TmaArgs {
    CUtensorMap m_int;   // spins, box (P, 8, 8, 1)
    CUtensorMap m_yh;    // spins, box (P, 1, 8, 1)
    CUtensorMap m_zh;    // spins, box (P, 8, 1, 1)
    CUtensorMap m_dmn;   // daemons, box (P, 8, 8, 1)
    CUtensorMap m_bond;  // bonds, box (P, 8, 8, 1)
    int8_t *spins;
    uint8_t *daemons;
    Geometry g;
    int S, R, r0, r1, parity;
    int ngroups, nb, ntiles, stages;  // nb = L / 8 tiles along y and z
    uint32_t stage_bytes, rep_bytes;  // shared memory per stage, per replica in a stage
    uint32_t key0, key1;
    const SweepParam *params;
    const int64_t *cursor;
    int64_t k;
    int *error;
    long long wait_limit;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    return done != 0;
}

// Bounded wait for phase `phase` of the mbarrier; false when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase, long long limit) {
    for (long long it = 0; it <= limit; ++it)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, int n,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(n), "r"(bar)
        : "memory");
}

struct TmaTile {
    int sample, ra, nrep, y0, z0;
};

__device__ __forceinline__ TmaTile tma_tile(const TmaArgs &a, int t) {
    TmaTile T;
    const int yb = t % a.nb;
    int rest = t / a.nb;
    const int zb = rest % a.nb;
    rest /= a.nb;
    const int grp = rest % a.ngroups;
    T.sample = rest / a.ngroups;
    T.ra = a.r0 + grp * kTmaRG;
    T.nrep = min(kTmaRG, a.r1 - T.ra);
    T.y0 = yb * kTmaT;
    T.z0 = zb * kTmaT;
    return T;
}

// Stage layout: per replica j of the tile [opp 8x8 | y-1 row x8 | y+8 row x8 |
// z-1 plane 8 rows | z+8 plane 8 rows | own spins 8x8 | own daemons 8x8] rows
// of P bytes, then the bonds 8x8. Every region is a multiple of 8 P bytes
// (128-byte aligned for P % 16 == 0).
__device__ __forceinline__ void tma_issue(const TmaArgs &a, uint8_t *stage, uint32_t bar, int t, bool refresh) {
    const TmaTile T = tma_tile(a, t);
    const Geometry &g = a.g;
    const int P = g.P, L = g.L, p = a.parity, op = 1 - p;
    const uint32_t tt = (uint32_t)(kTmaT * kTmaT * P), row8 = (uint32_t)(kTmaT * P);
    const uint32_t bytes = (uint32_t)T.nrep * ((refresh ? 2u : 3u) * tt + 4u * row8) + tt;
    mbar_expect_tx(bar, bytes);
    const int ym = (T.y0 + L - 1) % L, yp = (T.y0 + kTmaT) % L;
    const int zm = (T.z0 + L - 1) % L, zp = (T.z0 + kTmaT) % L;
    for (int j = 0; j < T.nrep; ++j) {
        const int gid = T.sample * a.R + T.ra + j;
        uint8_t *r = stage + (size_t)j * a.rep_bytes;
        const uint32_t s0 = smem_u32(r);
        tma_load_4d(s0, &a.m_int, 0, T.y0, T.z0, gid * 2 + op, bar);
        tma_load_4d(s0 + tt, &a.m_yh, 0, ym, T.z0, gid * 2 + op, bar);
        tma_load_4d(s0 + tt + row8, &a.m_yh, 0, yp, T.z0, gid * 2 + op, bar);
        tma_load_4d(s0 + tt + 2 * row8, &a.m_zh, 0, T.y0, zm, gid * 2 + op, bar);
        tma_load_4d(s0 + tt + 3 * row8, &a.m_zh, 0, T.y0, zp, gid * 2 + op, bar);
        tma_load_4d(s0 + tt + 4 * row8, &a.m_int, 0, T.y0, T.z0, gid * 2 + p, bar);
        if (!refresh) tma_load_4d(s0 + 2 * tt + 4 * row8, &a.m_dmn, 0, T.y0, T.z0, gid * 2 + p, bar);
    }
    tma_load_4d(smem_u32(stage + (size_t)kTmaRG * a.rep_bytes), &a.m_bond, 0, T.y0, T.z0, T.sample * 2 + p, bar);
}

__global__ void __launch_bounds__(kTmaThreads, 1) tma_half_kernel(const __grid_constant__ TmaArgs a) {
    extern __shared__ __align__(16) uint8_t sm_raw[];
    __shared__ __align__(8) uint64_t bars[kTmaMaxStages];
    // TMA destinations 128-byte aligned (128 bytes of slack are allocated)
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(sm_raw) + 127) & ~(uintptr_t)127);
    // parameters first: no kernel of a graph replay writes the table or the cursor
    const SweepParam prm = a.params[a.k + (a.cursor ? *a.cursor : 0)];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const bool refresh = prm.mode == kModeRefresh;
    const Geometry &g = a.g;
    const int P = g.P, L = g.L, p = a.parity;
    const int n_my = a.ntiles > (int)blockIdx.x ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) mbar_init(smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int s = 0; s < a.stages && s < n_my; ++s)
            tma_issue(a, sm + (size_t)s * a.stage_bytes, smem_u32(&bars[s]), blockIdx.x + s * gridDim.x, refresh);

    const int chunks = P / 16;  // 16-byte words of a row (4 sites each per 32-bit lane)
    const FastDiv div_chunks = make_fastdiv_dev((uint32_t)chunks);
    const uint32_t tt = (uint32_t)(kTmaT * kTmaT * P), row8 = (uint32_t)(kTmaT * P);
    for (int i = 0; i < n_my; ++i) {
        const int s = i % a.stages;
        const uint32_t phase = (uint32_t)((i / a.stages) & 1);
        const bool ok = mbar_wait_bounded(smem_u32(&bars[s]), phase, a.wait_limit);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicExch(a.error, 2);
                // loads still in flight: tiles i .. min(i + stages, n_my) - 1 (bounded)
                for (int q = i; q < n_my && q < i + a.stages; ++q)
                    mbar_wait_bounded(smem_u32(&bars[q % a.stages]), (uint32_t)((q / a.stages) & 1), a.wait_limit);
            }
            __syncthreads();
            return;
        }
        const int t = blockIdx.x + i * gridDim.x;
        const TmaTile T = tma_tile(a, t);
        const uint8_t *stage = sm + (size_t)s * a.stage_bytes;
        const uint8_t *bonds = stage + (size_t)kTmaRG * a.rep_bytes;
        const int items = T.nrep * kTmaT * kTmaT * chunks;
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const uint32_t rq = fdiv((uint32_t)it, div_chunks);
            const int c = it - (int)(rq * (uint32_t)chunks);
            const int j = (int)(rq >> 6), row = (int)(rq & 63), zz = row >> 3, yy = row & 7;
            const uint8_t *r = stage + (size_t)j * a.rep_bytes;
            const int8_t *opp = reinterpret_cast<const int8_t *>(r);
            const int8_t *O_row = opp + row * P;
            const int8_t *yp_row = yy < 7 ? O_row + P : opp + tt + row8 + zz * P;
            const int8_t *ym_row = yy > 0 ? O_row - P : opp + tt + zz * P;
            const int8_t *zp_row = zz < 7 ? O_row + 8 * P : opp + tt + 3 * row8 + yy * P;
            const int8_t *zm_row = zz > 0 ? O_row - 8 * P : opp + tt + 2 * row8 + yy * P;
            const int y = T.y0 + yy, z = T.z0 + zz, o = (p + y + z) & 1;
            const int b0 = c * 16;
            uint32_t Bw[4], O[4], Oyp[4], Oym[4], Ozp[4], Ozm[4], S[4], D[4];
            load_words<4>(bonds + row * P + b0, Bw);
            load_words<4>(O_row + b0, O);
            load_words<4>(yp_row + b0, Oyp);
            load_words<4>(ym_row + b0, Oym);
            load_words<4>(zp_row + b0, Ozp);
            load_words<4>(zm_row + b0, Ozm);
            load_words<4>(r + tt + 4 * row8 + row * P + b0, S);
            if (!refresh) load_words<4>(r + 2 * tt + 4 * row8 + row * P + b0, D);
            uint32_t edge = 0, first = 0, last = 0;
            if (o == 0) {
                if (b0 == 0) last = (uint8_t)O_row[g.Lh - 1];
                else edge = (uint8_t)O_row[b0 - 1];
            } else {
                if (b0 + 16 <= g.Lh - 1) edge = (uint8_t)O_row[b0 + 16];
                else first = (b0 == 0) ? (O[0] & 0xFFu) : (uint8_t)O_row[0];
            }
            uint32_t xp[4], xm[4];
            x_neighbours<4>(O, o, b0, g.Lh, edge, first, last, xp, xm);
            const uint32_t gid = (uint32_t)(T.sample * a.R + T.ra + j);
            const uint32_t quad0 = (uint32_t)((((int64_t)p * L + z) * L + y) * g.W + c * 4);
#pragma unroll
            for (int jw = 0; jw < 4; ++jw) {
                const uint32_t valid = valid_mask(b0, jw, g.Lh);
                if (refresh) {  // fresh daemons of this parity before its half-sweep (Sec. 2.7)
                    const uint4 w = philox4x32_10(make_uint4(quad0 + jw, (uint32_t)prm.t, (gid << 2) | kTagDaemon,
                                                             (uint32_t)((uint64_t)prm.t >> 32)),
                                                  a.key0, a.key1);
                    D[jw] = (daemon_from_uniform(w.x, prm.th0, prm.th1, prm.th2) |
                             (daemon_from_uniform(w.y, prm.th0, prm.th1, prm.th2) << 8) |
                             (daemon_from_uniform(w.z, prm.th0, prm.th1, prm.th2) << 16) |
                             (daemon_from_uniform(w.w, prm.th0, prm.th1, prm.th2) << 24)) & valid;
                }
                const uint32_t u32 = unsatisfied_count(Bw[jw], S[jw], xp[jw], xm[jw], Oyp[jw], Oym[jw], Ozp[jw],
                                                       Ozm[jw]);
                const uint32_t am = creutz4(u32, D[jw], valid);
                S[jw] ^= am & 0xFEFEFEFEu;
            }
            const int64_t goff = ((int64_t)gid * 2 + p) * g.half + ((int64_t)z * L + y) * P + b0;
            store_words<4>(a.spins + goff, S);
            store_words<4>(a.daemons + goff, D);
        }
        __syncthreads();  // the stage is free again
        if (threadIdx.x == 0 && i + a.stages < n_my) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_issue(a, sm + (size_t)s * a.stage_bytes, smem_u32(&bars[s]), blockIdx.x + (i + a.stages) * gridDim.x,
                      refresh);
        }
    }
}

bool tma_supported(const Geometry &g, int gamma, int walkers) {
    return g.P % 16 == 0 && g.P <= 256 && g.L % kTmaT == 0 && gamma == 1 && !walkers;
}

int tma_stages(const Geometry &g);
size_t tma_smem_bytes(const Geometry &g, int stages);

static uint32_t tma_rep_bytes(const Geometry &g) { return (uint32_t)(3 * kTmaT * kTmaT + 4 * kTmaT) * g.P; }
static uint32_t tma_stage_bytes(const Geometry &g) { return kTmaRG * tma_rep_bytes(g) + kTmaT * kTmaT * g.P; }

// Tensor maps of a handle's arrays (the driver's encoder through the runtime's
// entry-point query, so that no driver library is linked).
cudaError_t tma_encode(TmaMaps &m, int8_t *spins, uint8_t *daemons, const uint8_t *bonds, const Geometry &g, int S,
                       int R) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (!fn || q != cudaDriverEntryPointSuccess) return cudaErrorNotSupported;
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const cuuint32_t elem[4] = {1, 1, 1, 1};
    auto make = [&](CUtensorMap *map, void *base, uint64_t halves, uint32_t by, uint32_t bz) {
        const cuuint64_t dims[4] = {(cuuint64_t)g.P, (cuuint64_t)g.L, (cuuint64_t)g.L, (cuuint64_t)halves};
        const cuuint64_t strides[3] = {(cuuint64_t)g.P, (cuuint64_t)g.L * g.P, (cuuint64_t)g.half};
        const cuuint32_t box[4] = {(cuuint32_t)g.P, by, bz, 1};
        return encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, base, dims, strides, box, elem,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    };
    const uint64_t nrep = 2ull * S * R;
    if (make(&m.m_int, spins, nrep, kTmaT, kTmaT) != CUDA_SUCCESS ||
        make(&m.m_yh, spins, nrep, 1, kTmaT) != CUDA_SUCCESS ||
        make(&m.m_zh, spins, nrep, kTmaT, 1) != CUDA_SUCCESS ||
        make(&m.m_dmn, daemons, nrep, kTmaT, kTmaT) != CUDA_SUCCESS ||
        make(&m.m_bond, const_cast<uint8_t *>(bonds), 2ull * S, kTmaT, kTmaT) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    m.valid = true;
    return cudaSuccess;
}

size_t tma_smem_bytes(const Geometry &g, int stages) { return (size_t)stages * tma_stage_bytes(g) + 128; }

// CTAs of the persistent grid that fit on the device at once (0 on error).
int tma_max_ctas(const Geometry &g, int sm_count) {
    const int stages = tma_stages(g);
    if (stages < 2) return 0;
    const size_t smem = tma_smem_bytes(g, stages);
    if (cudaFuncSetAttribute(tma_half_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tma_half_kernel, kTmaThreads, smem) != cudaSuccess)
        return 0;
    return per_sm * sm_count;
}

int tma_stages(const Geometry &g) {
    const int s = (int)((size_t)(200 * 1024) / tma_stage_bytes(g));
    return std::max(0, std::min(kTmaMaxStages, s));
}

cudaError_t launch_tma_half(const TmaMaps &m, int8_t *spins, uint8_t *daemons, const Geometry &g, int S, int R,
                            int r0, int r1, int parity, uint32_t key0, uint32_t key1, const SweepParam *params,
                            const int64_t *cursor, int64_t k, int *error, long long wait_limit, int max_ctas,
                            bool pdl, cudaStream_t st) {
    const int stages = tma_stages(g);
    if (!m.valid || stages < 2 || r0 < 0 || r1 > R || r0 >= r1) return cudaErrorInvalidValue;
    TmaArgs a;
    a.m_int = m.m_int;
    a.m_yh = m.m_yh;
    a.m_zh = m.m_zh;
    a.m_dmn = m.m_dmn;
    a.m_bond = m.m_bond;
    a.spins = spins;
    a.daemons = daemons;
    a.g = g;
    a.S = S;
    a.R = R;
    a.r0 = r0;
    a.r1 = r1;
    a.parity = parity;
    a.ngroups = (r1 - r0 + kTmaRG - 1) / kTmaRG;
    a.nb = g.L / kTmaT;
    const int64_t ntiles = (int64_t)S * a.ngroups * a.nb * a.nb;
    if (ntiles >= (1ll << 31)) return cudaErrorInvalidValue;
    a.ntiles = (int)ntiles;
    a.stages = stages;
    a.rep_bytes = tma_rep_bytes(g);
    a.stage_bytes = tma_stage_bytes(g);
    a.key0 = key0;
    a.key1 = key1;
    a.params = params;
    a.cursor = cursor;
    a.k = k;
    a.error = error;
    a.wait_limit = wait_limit;
    const size_t smem = tma_smem_bytes(g, stages);
    cudaError_t e = cudaFuncSetAttribute(tma_half_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::max(1, std::min<int>(a.ntiles, max_ctas)));
    cfg.blockDim = dim3(kTmaThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tma_half_kernel, a);
}

}  // namespace micsa
