// onchip.cu -- persistent MicSA with the whole state of a run held in the
// shared memory of all SMs (byte layout), for lattices whose state fits there
// (L = 160 with two replicas: 20.5 MB of 34 MB).
//
// One cooperative launch runs K sweeps. CTA b owns a contiguous range
// [start, end) of the rows rho = z L + y of one sample (the sample's L^2 rows
// split evenly over k CTAs): the spins and daemons of both parities of all its
// replicas and the bonds of those rows live in its shared memory. Every
// neighbour row of an own row -- (z, y +- 1) and (z +- 1, y), periodic -- lies
// within L rows of the range in the periodic row space of the sample, so the
// rows [start - L, start) and [end, end + L) (mod L^2) are the halo. A
// half-sweep of parity p (Sec. 2.8 steps (i), (ii)):
//   1. wait until every CTA whose rows this one reads (and that reads this
//      one's rows) has finished the previous half-sweep -- one epoch flag per
//      CTA, written with release and polled with acquire semantics;
//   2. copy the halo rows of parity 1 - p from global memory (L2, bypassing L1);
//   3. update the own rows of parity p for every replica: Eq. (Creutz) with
//      Eq. (flip-OK) on four byte lanes per word, fresh daemons from the
//      library's Philox counters on refresh sweeps (Sec. 2.7);
//   4. write the updated spin rows to global memory (the copy the neighbours
//      read) and publish the epoch.
// The daemons go back to global memory at the end of the launch. Each wait is
// bounded: on time-out the CTA sets the error word and every CTA leaves its
// loop at its next wait. The spin, daemon and Philox arithmetic is that of the
// streaming kernel, so the results are bit-identical to every other engine.
#include <algorithm>
#include <vector>

#include "micsa_internal.h"
#include "../../include/micsa.h"

namespace micsa {

constexpr int kOcThreads = 512;
constexpr int kOcMaxNb = 16;     // neighbour CTAs per CTA
constexpr int kOcFlagStride = 32;  // one 128-byte line per epoch flag

struct OcRow {
    uint16_t s_yp, s_ym, s_zp, s_zm;  // neighbour slots: < qmax own row, else qmax + halo row
    uint16_t y, z;
};

struct OnchipArgs {
    int8_t *spins;          // [S][R][2][half] (global copy, kept current)
    uint8_t *daemons;       // [S][R][2][half]
    const uint8_t *bonds;   // [S][2][half]
    Geometry g;
    int S, R, k, qmax;      // k CTAs per sample, at most qmax rows each
    uint32_t key0, key1;
    const SweepParam *params;
    int64_t k0;             // first table entry of this launch
    int K;                  // sweeps in this launch
    unsigned *flags;        // [grid][kOcFlagStride], zero at launch
    int *error;             // set to 1 on a wait time-out
    const int16_t *nbrs;    // [grid][kOcMaxNb], -1 terminated
    long long wait_limit;   // polls per wait before giving up
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0: wait until every neighbour's epoch is >= target. Returns false on
// a time-out (recorded in *error) or when another CTA has recorded one.
__device__ bool oc_wait(const OnchipArgs &a, int b, unsigned target) {
    const int16_t *nb = a.nbrs + b * kOcMaxNb;
    for (int i = 0; i < kOcMaxNb; ++i) {
        const int n = nb[i];
        if (n < 0) break;
        long long it = 0;
        while (ld_acquire_gpu(a.flags + (size_t)n * kOcFlagStride) < target) {
            ++it;
            if ((it & 255) == 0 && *(volatile int *)a.error) return false;
            if (it > a.wait_limit) {
                atomicExch(a.error, 1);
                return false;
            }
        }
    }
    return true;
}

template <int NW>
__device__ __forceinline__ void ld_cg(const void *p, uint32_t (&w)[NW]) {
    if constexpr (NW == 4) {
        const uint4 v = __ldcg(reinterpret_cast<const uint4 *>(p));
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else if constexpr (NW == 2) {
        const uint2 v = __ldcg(reinterpret_cast<const uint2 *>(p));
        w[0] = v.x; w[1] = v.y;
    } else {
        w[0] = __ldcg(reinterpret_cast<const unsigned *>(p));
    }
}

template <int NW>
__global__ void __launch_bounds__(kOcThreads, 1) onchip_kernel(OnchipArgs a) {
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ int s_abort;
    const Geometry &g = a.g;
    const int b = blockIdx.x;
    if (b >= a.S * a.k) return;  // idle CTA: owns no rows and is nobody's neighbour
    const int sample = b / a.k, j = b - sample * a.k;
    const int64_t rows = (int64_t)g.L * g.L;
    const int start = (int)(j * rows / a.k), end = (int)((j + 1) * rows / a.k);
    const int Q = end - start, qmax = a.qmax, R = a.R, P = g.P, L = g.L;
    const bool halo = a.k > 1;

    // shared memory: spins [R][2][qmax][P], daemons [R][2][qmax][P], bonds
    // [2][qmax][P], halo [R][2L][P], row table [qmax]
    const size_t own = (size_t)R * 2 * qmax * P;
    int8_t *s_spin = reinterpret_cast<int8_t *>(sm);
    uint8_t *s_dmn = sm + own;
    uint8_t *s_bond = sm + 2 * own;
    int8_t *s_halo = reinterpret_cast<int8_t *>(sm + 2 * own + (size_t)2 * qmax * P);
    OcRow *s_row = reinterpret_cast<OcRow *>(sm + 2 * own + (size_t)2 * qmax * P +
                                             (halo ? (size_t)R * 2 * L * P : 0));

    // neighbour slots of the own rows
    auto slot = [&](int r2) -> uint16_t {
        if (r2 >= start && r2 < end) return (uint16_t)(r2 - start);
        const int dlo = (int)(((int64_t)r2 - (start - L) + rows) % rows);
        if (dlo < L) return (uint16_t)(qmax + dlo);
        return (uint16_t)(qmax + L + (int)(((int64_t)r2 - end + rows) % rows));
    };
    for (int q = threadIdx.x; q < Q; q += blockDim.x) {
        const int rho = start + q, z = rho / L, y = rho - z * L;
        OcRow e;
        e.y = (uint16_t)y;
        e.z = (uint16_t)z;
        e.s_yp = slot(y + 1 < L ? rho + 1 : rho - (L - 1));
        e.s_ym = slot(y > 0 ? rho - 1 : rho + (L - 1));
        e.s_zp = slot((int)((rho + L) % rows));
        e.s_zm = slot((int)((rho - L + rows) % rows));
        s_row[q] = e;
    }
    // own rows: spins, daemons, bonds (4-byte units; rows of one parity are contiguous)
    const int rowwords = P / 4;
    for (int r = 0; r < R; ++r)
        for (int par = 0; par < 2; ++par) {
            const int64_t gbase = (((int64_t)sample * R + r) * 2 + par) * g.half + (int64_t)start * P;
            const int64_t sbase = ((int64_t)r * 2 + par) * qmax * P;
            for (int w = threadIdx.x; w < Q * rowwords; w += blockDim.x) {
                reinterpret_cast<uint32_t *>(s_spin + sbase)[w] =
                    __ldcg(reinterpret_cast<const unsigned *>(a.spins + gbase) + w);
                reinterpret_cast<uint32_t *>(s_dmn + sbase)[w] =
                    __ldcg(reinterpret_cast<const unsigned *>(a.daemons + gbase) + w);
            }
        }
    for (int par = 0; par < 2; ++par) {
        const int64_t gbase = ((int64_t)sample * 2 + par) * g.half + (int64_t)start * P;
        for (int w = threadIdx.x; w < Q * rowwords; w += blockDim.x)
            reinterpret_cast<uint32_t *>(s_bond + (int64_t)par * qmax * P)[w] =
                __ldcg(reinterpret_cast<const unsigned *>(a.bonds + gbase) + w);
    }
    if (threadIdx.x == 0) s_abort = 0;
    __syncthreads();

    const int chunks = g.W / NW;
    const FastDiv div_chunks = make_fastdiv_dev((uint32_t)chunks);
    const FastDiv div_Q = make_fastdiv_dev((uint32_t)Q);
    const int items = R * Q * chunks;
    const int hunits = R * 2 * L * (P / (4 * NW));  // halo copy units of 4 NW bytes
    const FastDiv div_hrow = make_fastdiv_dev((uint32_t)(P / (4 * NW)));
    const FastDiv div_2L = make_fastdiv_dev((uint32_t)(2 * L));

    for (int e = 0; e < 2 * a.K; ++e) {
        const int p = e & 1, op = 1 - p;
        const SweepParam prm = a.params[a.k0 + (e >> 1)];
        const bool refresh = prm.mode == kModeRefresh;
        if (threadIdx.x == 0 && e > 0 && !oc_wait(a, b, (unsigned)e)) s_abort = 1;
        __syncthreads();
        if (s_abort) break;
        if (halo) {  // rows [start - L, start) and [end, end + L) of parity op, every replica
            for (int u = threadIdx.x; u < hunits; u += blockDim.x) {
                const int hr = (int)fdiv((uint32_t)u, div_hrow);  // (r, halo row)
                const int cw = u - hr * (P / (4 * NW));
                const int r = (int)fdiv((uint32_t)hr, div_2L), h = hr - r * 2 * L;
                const int rho = h < L ? (int)(((int64_t)start - L + h + rows) % rows)
                                      : (int)(((int64_t)end + (h - L)) % rows);
                const int64_t goff = (((int64_t)sample * R + r) * 2 + op) * g.half + (int64_t)rho * P + cw * 4 * NW;
                uint32_t w[NW];
                ld_cg<NW>(a.spins + goff, w);
                store_words<NW>(s_halo + ((int64_t)r * 2 * L + h) * P + cw * 4 * NW, w);
            }
            __syncthreads();
        }
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int rq = (int)fdiv((uint32_t)it, div_chunks);
            const int c = it - rq * chunks;
            const int r = (int)fdiv((uint32_t)rq, div_Q), q = rq - r * Q;
            const OcRow row = s_row[q];
            const int y = row.y, z = row.z;
            const int o = (p + y + z) & 1;
            const int b0 = c * 4 * NW;
            const int8_t *opp_own = s_spin + ((int64_t)r * 2 + op) * qmax * P;
            auto opp_row = [&](int s) -> const int8_t * {
                return s < qmax ? opp_own + (int64_t)s * P : s_halo + ((int64_t)r * 2 * L + (s - qmax)) * P;
            };
            const int8_t *oc = opp_own + (int64_t)q * P;
            int8_t *own_s = s_spin + (((int64_t)r * 2 + p) * qmax + q) * P;
            uint8_t *own_d = s_dmn + (((int64_t)r * 2 + p) * qmax + q) * P;
            uint32_t Bw[NW], O[NW], Oyp[NW], Oym[NW], Ozp[NW], Ozm[NW], S[NW], D[NW];
            load_words<NW>(s_bond + ((int64_t)p * qmax + q) * P + b0, Bw);
            load_words<NW>(oc + b0, O);
            load_words<NW>(opp_row(row.s_yp) + b0, Oyp);
            load_words<NW>(opp_row(row.s_ym) + b0, Oym);
            load_words<NW>(opp_row(row.s_zp) + b0, Ozp);
            load_words<NW>(opp_row(row.s_zm) + b0, Ozm);
            load_words<NW>(own_s + b0, S);
            if (!refresh) load_words<NW>(own_d + b0, D);
            uint32_t edge = 0, first = 0, last = 0;
            if (o == 0) {
                if (b0 == 0) last = (uint8_t)oc[g.Lh - 1];
                else edge = (uint8_t)oc[b0 - 1];
            } else {
                if (b0 + 4 * NW <= g.Lh - 1) edge = (uint8_t)oc[b0 + 4 * NW];
                else first = (b0 == 0) ? (O[0] & 0xFFu) : (uint8_t)oc[0];
            }
            uint32_t xp[NW], xm[NW];
            x_neighbours<NW>(O, o, b0, g.Lh, edge, first, last, xp, xm);
            const uint32_t gid = (uint32_t)(sample * R + r);
            const uint32_t quad0 = (uint32_t)((((int64_t)p * L + z) * L + y) * g.W + c * NW);
#pragma unroll
            for (int jw = 0; jw < NW; ++jw) {
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
            store_words<NW>(own_s + b0, S);
            store_words<NW>(own_d + b0, D);
            store_words<NW>(a.spins + (((int64_t)gid * 2 + p) * g.half + (int64_t)(start + q) * P + b0), S);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_gpu(a.flags + (size_t)b * kOcFlagStride, (unsigned)(e + 1));
        }
    }
    __syncthreads();
    if (s_abort) return;
    // daemons back to global memory (the spins are there already)
    for (int r = 0; r < R; ++r)
        for (int par = 0; par < 2; ++par) {
            const int64_t gbase = (((int64_t)sample * R + r) * 2 + par) * g.half + (int64_t)start * P;
            const int64_t sbase = ((int64_t)r * 2 + par) * qmax * P;
            for (int w = threadIdx.x; w < Q * rowwords; w += blockDim.x)
                reinterpret_cast<uint32_t *>(a.daemons + gbase)[w] =
                    reinterpret_cast<const uint32_t *>(s_dmn + sbase)[w];
        }
}

template <int NW>
static const void *onchip_fn() {
    return (const void *)onchip_kernel<NW>;
}

static const void *onchip_kernel_for(int nw) {
    return nw == 4 ? onchip_fn<4>() : nw == 2 ? onchip_fn<2>() : onchip_fn<1>();
}

size_t onchip_smem_bytes(const Geometry &g, int R, int k, int qmax) {
    const size_t own = (size_t)R * 2 * qmax * g.P;
    return 2 * own + (size_t)2 * qmax * g.P + (k > 1 ? (size_t)R * 2 * g.L * g.P : 0) + sizeof(OcRow) * qmax;
}

// Partition and neighbour table for S samples on up to `ctas` co-resident CTAs.
// Returns false if the lattice does not fit (shared memory, row slots,
// neighbour count).
bool onchip_plan(const Geometry &g, int S, int R, int ctas, int nw, OnchipPlan &plan) {
    if (g.L < 8 || S < 1 || ctas < S) return false;
    const int64_t rows = (int64_t)g.L * g.L;
    int k = ctas / S;
    if (k > rows / 2) k = (int)(rows / 2);
    const int qmax = (int)((rows + k - 1) / k);
    if (qmax + 2 * g.L > 65535) return false;  // 16-bit row slots
    const size_t smem = onchip_smem_bytes(g, R, k, qmax);
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return false;
    if (smem + 64 > (size_t)optin) return false;
    std::vector<int64_t> st(k + 1);
    for (int j = 0; j <= k; ++j) st[j] = j * rows / k;
    auto owner = [&](int64_t row) {
        return (int)(std::upper_bound(st.begin(), st.end(), row) - st.begin()) - 1;
    };
    std::vector<std::vector<int>> nb(k);
    if (k > 1)
        for (int j = 0; j < k; ++j)
            for (int i = 0; i < g.L; ++i) {
                const int o1 = owner(((st[j] - g.L + i) % rows + rows) % rows);
                const int o2 = owner((st[j + 1] + i) % rows);
                for (int o : {o1, o2})
                    if (o != j) {
                        if (std::find(nb[j].begin(), nb[j].end(), o) == nb[j].end()) nb[j].push_back(o);
                        if (std::find(nb[o].begin(), nb[o].end(), j) == nb[o].end()) nb[o].push_back(j);
                    }
            }
    plan.table.assign((size_t)S * k * kOcMaxNb, (int16_t)-1);
    for (int a = 0; a < S; ++a)
        for (int j = 0; j < k; ++j) {
            if ((int)nb[j].size() > kOcMaxNb) return false;
            for (size_t i = 0; i < nb[j].size(); ++i)
                plan.table[((size_t)a * k + j) * kOcMaxNb + i] = (int16_t)(a * k + nb[j][i]);
        }
    plan.k = k;
    plan.qmax = qmax;
    plan.grid = S * k;
    plan.nw = nw;
    plan.smem = smem;
    const void *fn = onchip_kernel_for(nw);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return false;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kOcThreads, smem) != cudaSuccess || per_sm < 1)
        return false;
    return true;
}

// A one-CTA kernel that runs the epoch wait on a flag nothing sets: the
// bounded-wait path of the engine, exercised without any fault.
__global__ void wait_selftest_kernel(unsigned *flag, int *error, long long wait_limit) {
    const int16_t nb[kOcMaxNb] = {0, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
    OnchipArgs a{};
    a.flags = flag;
    a.error = error;
    a.nbrs = nb;
    a.wait_limit = wait_limit;
    if (threadIdx.x == 0) oc_wait(a, 0, 1u);
}

cudaError_t launch_wait_selftest(unsigned *flag, int *error, long long wait_limit, cudaStream_t st) {
    wait_selftest_kernel<<<1, 32, 0, st>>>(flag, error, wait_limit);
    return cudaGetLastError();
}

size_t onchip_flag_words(int grid) { return (size_t)grid * kOcFlagStride; }
int onchip_max_neighbours() { return kOcMaxNb; }

cudaError_t launch_onchip(const OnchipPlan &plan, int8_t *spins, uint8_t *daemons, const uint8_t *bonds,
                          const Geometry &g, int S, int R, uint32_t key0, uint32_t key1, const SweepParam *params,
                          int64_t k0, int K, unsigned *flags, int *error, const int16_t *nbrs, long long wait_limit,
                          cudaStream_t st) {
    // the attribute is per function: another handle may have planned a smaller size
    cudaError_t e = cudaFuncSetAttribute(onchip_kernel_for(plan.nw), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)plan.smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(flags, 0, sizeof(unsigned) * onchip_flag_words(plan.grid), st);
    if (e != cudaSuccess) return e;
    OnchipArgs a{};
    a.spins = spins;
    a.daemons = daemons;
    a.bonds = bonds;
    a.g = g;
    a.S = S;
    a.R = R;
    a.k = plan.k;
    a.qmax = plan.qmax;
    a.key0 = key0;
    a.key1 = key1;
    a.params = params;
    a.k0 = k0;
    a.K = K;
    a.flags = flags;
    a.error = error;
    a.nbrs = nbrs;
    a.wait_limit = wait_limit;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)plan.grid);
    cfg.blockDim = dim3(kOcThreads);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs co-resident: the epoch waits need it
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *kargs[] = {&a};
    return cudaLaunchKernelExC(&cfg, onchip_kernel_for(plan.nw), kargs);
}

}  // namespace micsa
