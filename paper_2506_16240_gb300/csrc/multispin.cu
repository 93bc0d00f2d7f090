// multispin.cu -- MicSA with multispin coding (the Boolean-only update the
// paper describes for its CUDA code, App. B and Sec. 2.5) in two forms: the
// shared-memory resident kernel for lattices with L <= 32 (first part of this
// file) and the bit planes in HBM for L a multiple of 32, with gamma daemon
// families and walkers (second part).
//
// A CTA converts one replica from the global byte layout into bit planes in
// shared memory, runs a block of sweeps there, and converts back. Bit plane
// words: for parity p, row y and half-row index i, bit z of word (p, y, i)
// belongs to the site x = 2i + ((p + y + z) & 1), y, z of parity p (the same
// site the byte layout keeps at row (z, y), byte i). Planes: spin sign (1 = -1),
// daemon bits m0 and m1, and six bond planes (bit set <=> J = -1) for +x, +y,
// +z, -x, -y, -z.
//
// Neighbours of the 32 sites of word (p, y, i) in the opposite parity:
//   +-y: word (1-p, y+-1, i)                    (same x offset)
//   +-z: word (1-p, y, i) rotated by one bit    (same x, periodic in L bits)
//   +x:  bits with x offset 0 take word (1-p, y, i), offset 1 take (1-p, y, i+1)
//   -x:  offset 0 take (1-p, y, i-1), offset 1 take (1-p, y, i)
// The number u of unsatisfied bonds (J s s_nb = -1) is summed bit-sliced; the
// move of Eq. (Creutz) with Eq. (flip-OK) is accept <=> 3 <= u + m <= 6,
// m' = u + m - 3 (dH = 12 - 4u), evaluated with Boolean operations only. The
// daemon refresh draws the same Philox words as every other kernel, so the
// results are bit-identical to them.
#include <algorithm>

#include "sweep_body.cuh"
#include "msg_body.cuh"
#include "../../include/micsa.h"

namespace micsa {

constexpr int kMsThreads = 512;  // >= L * L / 2 words of one parity for L <= 32
constexpr int kMsPoolMaxR = MICSA_POOL_MAX_REPLICAS;

// bit-plane words per parity and plane
__host__ __device__ __forceinline__ int ms_words(int L) { return L * (L / 2); }

size_t multispin_smem_bytes(const Geometry &g) {
    if (g.L > 32) return 0;
    return sizeof(uint32_t) * 9 * 2 * (size_t)ms_words(g.L);
}

struct MsPlanes {
    uint32_t *s, *m0, *m1, *b;  // each [2][L][Lh]; b: [6][2][L][Lh]
    int L, Lh, n;               // n = words per parity
    __device__ __forceinline__ int idx(int p, int y, int i) const { return (p * L + y) * Lh + i; }
    __device__ __forceinline__ uint32_t &bond(int k, int p, int y, int i) const { return b[k * 2 * n + idx(p, y, i)]; }
};

__device__ __forceinline__ uint32_t rot_up(uint32_t v, int L, uint32_t mask) {  // bit z <- bit z-1
    return L == 32 ? __funnelshift_l(v, v, 1) : (((v << 1) | (v >> (L - 1))) & mask);
}
__device__ __forceinline__ uint32_t rot_down(uint32_t v, int L, uint32_t mask) {  // bit z <- bit z+1
    return L == 32 ? __funnelshift_r(v, v, 1) : (((v >> 1) | (v << (L - 1))) & mask);
}

// Byte layout (global) -> bit planes. One warp per (parity, y, word q of the
// row) -- the four sites i = 4q .. 4q+3 -- and one lane per z: a lane loads
// the byte words of row (z, y) and the warp votes each bit plane together.
__device__ void ms_pack(const MsPlanes &P, const Geometry &g, const int8_t *spins, const uint8_t *daemons,
                        const uint8_t *bonds) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int items = 2 * g.L * g.W;
    for (int it = warp; it < items; it += nwarps) {
        const int q = it % g.W;
        const int y = (it / g.W) % g.L;
        const int p = it / (g.W * g.L);
        uint32_t S = 0, D = 0, B = 0;
        if (lane < g.L) {
            const int64_t off = (int64_t)p * g.half + ((int64_t)lane * g.L + y) * g.P + 4 * q;
            S = *reinterpret_cast<const uint32_t *>(spins + off);
            D = *reinterpret_cast<const uint32_t *>(daemons + off);
            B = *reinterpret_cast<const uint32_t *>(bonds + off);
        }
        // lane 9 l + j (j < 9) stores plane j of word i = 4q + l: spin, m0, m1, bonds 0..5
        uint32_t mine = 0;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const uint32_t v[9] = {__ballot_sync(0xFFFFFFFFu, (S >> (8 * l + 7)) & 1u),
                                   __ballot_sync(0xFFFFFFFFu, (D >> (8 * l)) & 1u),
                                   __ballot_sync(0xFFFFFFFFu, (D >> (8 * l + 1)) & 1u),
                                   __ballot_sync(0xFFFFFFFFu, (B >> (8 * l)) & 1u),
                                   __ballot_sync(0xFFFFFFFFu, (B >> (8 * l + 1)) & 1u),
                                   __ballot_sync(0xFFFFFFFFu, (B >> (8 * l + 2)) & 1u),
                                   __ballot_sync(0xFFFFFFFFu, (B >> (8 * l + 3)) & 1u),
                                   __ballot_sync(0xFFFFFFFFu, (B >> (8 * l + 4)) & 1u),
                                   __ballot_sync(0xFFFFFFFFu, (B >> (8 * l + 5)) & 1u)};
#pragma unroll
            for (int j = 0; j < 9; ++j)
                if (lane == 9 * l + j || (l == 3 && lane + 32 == 9 * l + j)) mine = v[j];
            if (l == 2) {  // lanes 0..26 hold words 0..2; store them, then reuse lanes for word 3
                const int j = lane % 9, li = lane / 9, i = 4 * q + li;
                if (lane < 27 && i < g.Lh) {
                    const int w = P.idx(p, y, i);
                    uint32_t *dst = j == 0 ? &P.s[w] : j == 1 ? &P.m0[w] : j == 2 ? &P.m1[w] : &P.bond(j - 3, p, y, i);
                    *dst = mine;
                }
                mine = 0;
            }
        }
        {
            // word 3: planes 0..4 went to lanes 27..31, planes 5..8 to lanes 0..3
            const int j = lane >= 27 ? lane - 27 : lane + 5, i = 4 * q + 3;
            if ((lane >= 27 || lane < 4) && i < g.Lh) {
                const int w = P.idx(p, y, i);
                uint32_t *dst = j == 0 ? &P.s[w] : j == 1 ? &P.m0[w] : j == 2 ? &P.m1[w] : &P.bond(j - 3, p, y, i);
                *dst = mine;
            }
        }
    }
}

// Bit planes -> byte layout (spins and daemons; bonds never change). Same
// warp/lane mapping as ms_pack.
__device__ void ms_unpack(const MsPlanes &P, const Geometry &g, int8_t *spins, uint8_t *daemons) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int items = 2 * g.L * g.W;
    for (int it = warp; it < items; it += nwarps) {
        const int q = it % g.W;
        const int y = (it / g.W) % g.L;
        const int p = it / (g.W * g.L);
        if (lane >= g.L) continue;
        uint32_t S = 0, D = 0;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int i = 4 * q + l;
            if (i >= g.Lh) break;
            const int w = P.idx(p, y, i);
            S |= (((P.s[w] >> lane) & 1u) ? 0xFFu : 0x01u) << (8 * l);
            D |= (((P.m0[w] >> lane) & 1u) | (((P.m1[w] >> lane) & 1u) << 1)) << (8 * l);
        }
        const uint32_t valid = valid_mask(4 * q, 0, g.Lh);
        const int64_t off = (int64_t)p * g.half + ((int64_t)lane * g.L + y) * g.P + 4 * q;
        *reinterpret_cast<uint32_t *>(spins + off) = S & valid;
        *reinterpret_cast<uint32_t *>(daemons + off) = D & valid;
    }
}

// Daemon bit planes of words (p, y, i), i = 4q .. 4q+3, for the refresh at
// sweep t. Lane z draws the Philox block of site z -- quad = ((p L + z) L + y) W
// + q, lane i & 3 of the block for word i (the library's counter contract) --
// and the warp votes the two daemon bit planes of the four words.
__device__ __forceinline__ void ms_refresh_warp(const MsPlanes &P, const Geometry &g, int p, int y, int q,
                                                uint32_t gid, const RoundKeys &rk, int64_t t, const CutsGt &cut) {
    const int lane = threadIdx.x & 31;
    uint4 w = make_uint4(0, 0, 0, 0);  // lanes z >= L: u = 0 is below every cut point, m = 0
    if (lane < g.L) {
        const uint32_t quad = (uint32_t)((((int64_t)p * g.L + lane) * g.L + y) * g.W + q);
        w = philox_wide(make_uint4(quad, (uint32_t)t, (gid << 2) | kTagDaemon, (uint32_t)((uint64_t)t >> 32)), rk);
    }
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
    // planes (m0, m1) of the four words; lane j < 8 stores plane j & 1 of word j >> 1
    uint32_t mine = 0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const bool g0 = u[l] > cut.c0m, g1 = u[l] > cut.c1m, g2 = u[l] > cut.c2m;
        const uint32_t a = __ballot_sync(0xFFFFFFFFu, g0 ^ g1 ^ g2);
        const uint32_t c = __ballot_sync(0xFFFFFFFFu, g1);
        if (lane == 2 * l) mine = a;
        if (lane == 2 * l + 1) mine = c;
    }
    const int i = 4 * q + (lane >> 1);
    if (lane < 8 && i < g.Lh) {
        const int wi = P.idx(p, y, i);
        ((lane & 1) ? P.m1 : P.m0)[wi] = mine;
    }
}

// Word indices of one thread's site word (y, i) for parity p and its
// opposite-parity neighbours, computed once per unit (L <= 32 gives at most
// L * L / 2 <= 512 words per parity, one per thread).
struct MsItem {
    int own, oc, oip, oim, oyp, oym;
    uint32_t M;  // bits whose site has x offset 1
};

__device__ __forceinline__ MsItem ms_item(const MsPlanes &P, int p, int y, int i, uint32_t mask) {
    const int L = P.L, Lh = P.Lh, o = 1 - p;
    const int yp = (y + 1 == L) ? 0 : y + 1, ym = (y == 0) ? L - 1 : y - 1;
    const int ip = (i + 1 == Lh) ? 0 : i + 1, im = (i == 0) ? Lh - 1 : i - 1;
    MsItem it;
    it.own = P.idx(p, y, i);
    it.oc = P.idx(o, y, i);
    it.oip = P.idx(o, y, ip);
    it.oim = P.idx(o, y, im);
    it.oyp = P.idx(o, yp, i);
    it.oym = P.idx(o, ym, i);
    it.M = (((p + y) & 1) ? 0x55555555u : 0xAAAAAAAAu) & mask;
    return it;
}

// The elementary move on the 32 sites of one word (Eq. Creutz, Eq. flip-OK).
__device__ __forceinline__ void ms_update(const MsPlanes &P, const MsItem &it, int L, uint32_t mask) {
    const uint32_t *bp = P.b + it.own;  // bond plane k of this word at bp[k * 2n]
    const int stride = 2 * P.n;
    const uint32_t Oc = P.s[it.oc];
    const uint32_t nxp = (Oc & ~it.M) | (P.s[it.oip] & it.M);
    const uint32_t nxm = (P.s[it.oim] & ~it.M) | (Oc & it.M);
    const uint32_t nzp = rot_down(Oc, L, mask);
    const uint32_t nzm = rot_up(Oc, L, mask);
    const uint32_t sg = P.s[it.own];
    // unsatisfied bond indicators: j ^ s ^ s_nb
    const uint32_t q0 = sg ^ nxp ^ bp[0];
    const uint32_t q1 = sg ^ P.s[it.oyp] ^ bp[stride];
    const uint32_t q2 = sg ^ nzp ^ bp[2 * stride];
    const uint32_t q3 = sg ^ nxm ^ bp[3 * stride];
    const uint32_t q4 = sg ^ P.s[it.oym] ^ bp[4 * stride];
    const uint32_t q5 = sg ^ nzm ^ bp[5 * stride];
    // u = q0 + ... + q5 (bit-sliced, three planes)
    const uint32_t s1 = q0 ^ q1 ^ q2, c1 = (q0 & q1) | (q2 & (q0 ^ q1));
    const uint32_t s2 = q3 ^ q4 ^ q5, c2 = (q3 & q4) | (q5 & (q3 ^ q4));
    const uint32_t u0 = s1 ^ s2, k = s1 & s2;
    const uint32_t u1 = c1 ^ c2 ^ k, u2 = (c1 & c2) | (k & (c1 ^ c2));
    // v = u + m (four planes)
    const uint32_t m0 = P.m0[it.own], m1 = P.m1[it.own];
    const uint32_t v0 = u0 ^ m0, k0 = u0 & m0;
    const uint32_t v1 = u1 ^ m1 ^ k0, k1 = (u1 & m1) | (k0 & (u1 ^ m1));
    const uint32_t v2 = u2 ^ k1, v3 = u2 & k1;
    // 3 <= v <= 6  <=>  v3 == 0 and v2 != (v1 & v0); then m' = v - 3
    const uint32_t acc = (v2 ^ (v1 & v0)) & ~v3 & mask;
    P.m0[it.own] = (m0 & ~acc) | (~v0 & acc);
    P.m1[it.own] = (m1 & ~acc) | (v2 & (v1 | v0) & acc);
    P.s[it.own] = sg ^ acc;
}

__device__ __forceinline__ void ms_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void ms_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <bool POOL>
__global__ void __launch_bounds__(kMsThreads, 2) multispin_kernel(ResidentArgs A) {
    ms_wait();
    ms_release();
    extern __shared__ __align__(16) uint32_t msm[];
    __shared__ int s_unit;
    __shared__ long long s_red[2][kMsThreads / 32];
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
            if (t0 >= n_sweeps) {
                __syncthreads();
                continue;
            }
        }
        const int n = ms_words(g.L);
        MsPlanes P{msm, msm + 2 * n, msm + 4 * n, msm + 6 * n, g.L, g.Lh, n};
        const uint32_t mask = g.L == 32 ? 0xFFFFFFFFu : ((1u << g.L) - 1u);
        ms_pack(P, g, U.spins, U.daemons, U.bonds);
        const bool has_item = threadIdx.x < n;  // n <= blockDim for L <= 32
        const int iy = has_item ? (int)threadIdx.x / g.Lh : 0, ix = has_item ? (int)threadIdx.x - iy * g.Lh : 0;
        const MsItem item[2] = {ms_item(P, 0, iy, ix, mask), ms_item(P, 1, iy, ix, mask)};
        const RoundKeys rk = round_keys(key0, key1);
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
                if (refresh) {  // fresh daemons of parity p before its half-sweep (Sec. 2.7)
                    const CutsGt cut = make_cuts_gt(th0, th1, th2);
                    const int items = g.L * g.W;
                    for (int it = threadIdx.x >> 5; it < items; it += blockDim.x >> 5)
                        ms_refresh_warp(P, g, p, it / g.W, it % g.W, (uint32_t)U.gid, rk, t, cut);
                    __syncthreads();
                }
                if (has_item) ms_update(P, item[p], g.L, mask);
                __syncthreads();
            }
            t_end = t + 1;
        }
        ms_unpack(P, g, U.spins, U.daemons);

        if (POOL) {
            // exact energy (even sites: 2u - 6 each) and daemon energy from the planes
            long long e = 0, a = 0;
            for (int it = threadIdx.x; it < n; it += blockDim.x) {
                const int y = it / g.Lh, i = it - y * g.Lh;
                const int yp = (y + 1 == g.L) ? 0 : y + 1, ym = (y == 0) ? g.L - 1 : y - 1;
                const int ip = (i + 1 == g.Lh) ? 0 : i + 1, im = (i == 0) ? g.Lh - 1 : i - 1;
                const uint32_t Oc = P.s[P.idx(1, y, i)];
                const uint32_t M = ((y & 1) ? 0x55555555u : 0xAAAAAAAAu) & mask;
                const uint32_t nb[6] = {(Oc & ~M) | (P.s[P.idx(1, y, ip)] & M), P.s[P.idx(1, yp, i)],
                                        rot_down(Oc, g.L, mask), (P.s[P.idx(1, y, im)] & ~M) | (Oc & M),
                                        P.s[P.idx(1, ym, i)], rot_up(Oc, g.L, mask)};
                const uint32_t sg = P.s[P.idx(0, y, i)];
                int usum = 0;
#pragma unroll
                for (int kk = 0; kk < 6; ++kk) usum += __popc((sg ^ nb[kk] ^ P.bond(kk, 0, y, i)) & mask);
                e += 2 * usum - 6 * g.L;
                a += 4 * (__popc(P.m0[P.idx(0, y, i)]) + 2 * __popc(P.m1[P.idx(0, y, i)]) +
                          __popc(P.m0[P.idx(1, y, i)]) + 2 * __popc(P.m1[P.idx(1, y, i)]));
            }
            e = __reduce_add_sync(0xFFFFFFFFu, (int)e);
            a = __reduce_add_sync(0xFFFFFFFFu, (int)a);
            if ((threadIdx.x & 31) == 0) {
                s_red[0][threadIdx.x >> 5] = e;
                s_red[1][threadIdx.x >> 5] = a;
            }
            __syncthreads();
            const int cell = U.slot * kMsPoolMaxR + U.gid;
            const int64_t rows = (int64_t)A.max_jobs * kMsPoolMaxR;
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
                    best[site] = ((P.s[P.idx(par, y, x >> 1)] >> z) & 1u) ? (int8_t)-1 : (int8_t)1;
                }
            }
        }
        __syncthreads();  // the planes are reused by the next unit
    }
}

cudaError_t launch_multispin(const ResidentArgs &a, bool pool, size_t smem, int grid, bool pdl, cudaStream_t st) {
    const void *fn = pool ? (const void *)multispin_kernel<true> : (const void *)multispin_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kMsThreads);
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

int multispin_blocks_per_sm(bool pool, size_t smem) {
    const void *fn = pool ? (const void *)multispin_kernel<true> : (const void *)multispin_kernel<false>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kMsThreads, smem) != cudaSuccess) return 0;
    return n;
}

}  // namespace micsa

// ===================================================================
// Global-memory multispin engine (L a multiple of 32): the lattice lives in
// bit planes in HBM for the whole run. Plane word (p, zw, y, i) holds, in bit
// b, the site x = 2i + ((p + y + z) & 1), y, z = 32 zw + b of parity p (the
// site the byte layout keeps at row (z, y), byte i). Word index within a
// parity plane: (zw * L + y) * Lh + i, WP = L^3 / 64 words per parity (the
// pool's bit-plane jobs, any even L > 32, use the same layout with ceil(L / 32)
// z words, the last one partial, and rows of P = 4 ceil(Lh / 4) words, the words
// from Lh on padding). Per
// replica the planes are [spin | m0 | m1][parity][WP]; per sample the bond
// planes are [6][parity][WP] (bit set <=> J = -1, order +x +y +z -x -y -z).
//
// With gamma daemon families (Sec. 2.8) the daemon planes are
// [buffer][family][m0 | m1][parity] after the two spin planes; family alpha of
// replica gid draws with Philox id gid * gamma + alpha. With walkers (Sec. 2.6)
// there are two buffers: the sweeps of timestep t use buffer t & 1 and the
// wandering step after timestep t gathers buffer t & 1 into buffer (t + 1) & 1
// (a permutation of the daemon bits, so out of place is race-free).
//
// A thread owns NW consecutive words i = i0 .. i0+NW-1 of one (zw, y) and runs
// the replicas r = blockIdx.y * rpt .. of its sample over them, so one load
// of the bond words serves rpt replicas. The z neighbours of bit 31 (bit 0)
// sit in bit 0 (bit 31) of the word of z-word zw + 1 (zw - 1): funnel shifts.
// A refresh draws the Philox block of quad ((p L + z) L + y) W + i/4 for
// every z (the library's counter contract); the 4 / NW lanes that share a
// block of words split the 32 z between them and OR their partial planes
// together with shuffles.
// ===================================================================
namespace micsa {

struct MsgArgs {
    uint32_t *planes;        // [S*R][NP][WP], NP = 2 + 4 gamma (x 2 buffers with walkers)
    const uint32_t *bonds;   // [S][6][2][WP]
    int L, Lh, nzw, W4;      // W4 = Lh / 4 Philox blocks per row
    int64_t WP;
    int S, R, r0, r1, rpt, parity;  // replicas [r0, r1) of every sample, rpt per thread
    int gamma, walkers, np;         // daemon families, two daemon buffers, planes per replica
    uint32_t key0, key1;
    const SweepParam *params;
    const int64_t *cursor;
    int64_t k;
    FastDiv div_groups, div_L;  // thread index -> (zw, y, word group)
};

// MINB: minimum resident blocks of 128 per SM the register allocation must
// allow (4: the default, at most 128 registers; 5: the register-capped
// variant, at most 102).
template <int NW, int MINB, bool METRO = false>
__global__ void __launch_bounds__(128, MINB) msg_half_kernel(MsgArgs a) {
    // parameters first: no kernel of a graph replay writes the table or the cursor
    const int64_t kidx = a.k + (a.cursor ? *a.cursor : 0);
    const SweepParam prm = a.params[kidx];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // grid: x covers the L * nzw * Lh / NW threads of one sample exactly (a
    // multiple of 128 for L % 32 == 0), y the replica groups, z the samples
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int sample = (int)blockIdx.z;
    const uint32_t rowi = fdiv(tid, a.div_groups);
    const int ig = (int)(tid - rowi * a.div_groups.d);
    const uint32_t zw_u = fdiv(rowi, a.div_L);
    const int y = (int)(rowi - zw_u * a.div_L.d);
    const MsgLattice lat{a.planes + (int64_t)sample * a.R * a.np * a.WP, a.bonds + (int64_t)sample * 12 * a.WP,
                         a.L, a.Lh, a.nzw, a.W4, a.WP, a.np, a.gamma, a.walkers, (int64_t)sample * a.R,
                         a.key0, a.key1, a.Lh};
    const int r_begin = a.r0 + (int)blockIdx.y * a.rpt;
    msg_update<NW, false, METRO>(lat, prm, a.parity, (int)zw_u, y, ig, r_begin, min(a.r1, r_begin + a.rpt));
}

// bytes <-> planes. One thread per plane word (n_rep replicas, two parities,
// WP words); the 32 bits of a word are the 32 z of one (y, i). Daemons: the
// gamma families of buffer buf.
__global__ void msg_convert_state_kernel(uint32_t *planes, int8_t *spins, uint8_t *daemons, Geometry g,
                                         int64_t n_rep, int64_t WP, int gamma, int np, int buf, bool to_planes) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= n_rep * 2 * WP) return;
    const int64_t rep = tid / (2 * WP);
    const int64_t rem = tid - rep * 2 * WP;
    const int p = (int)(rem / WP);
    msg_convert_word(planes, spins, daemons, g, WP, gamma, np, buf, to_planes, rep, p, rem - (int64_t)p * WP);
}

// Wandering step on the daemon planes (Sec. 2.6), out of place: after timestep
// t every site of parity q = t & 1 exchanges its walker of family alpha with
// its neighbour along direction alpha mod 6 (+x, +y, +z, -x, -y, -z). A site
// of parity q takes the walker of its neighbour at +d, a site of parity 1 - q
// that of its neighbour at -d; the neighbour word is assembled from the other
// parity's plane exactly as the spin neighbours of the update. One thread per
// output word (replica, family, parity, word), both daemon bits.
// Grid: x over the WP words, y over (replica of [r0, r1), family, parity), z
// over samples.
__global__ void msg_wander_kernel(uint32_t *planes, Geometry g, int R, int r0, int gamma, int np, uint32_t WP,
                                  FastDiv div_Lh, FastDiv div_L, const SweepParam *params, const int64_t *cursor,
                                  int64_t k) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int64_t t = params[k + (cursor ? *cursor : 0)].t;
    const int q = (int)(t & 1), src = (int)(t & 1), dst = 1 - src;
    const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= WP) return;
    const int P = (int)(blockIdx.y & 1);
    const int fr = (int)(blockIdx.y >> 1);
    const int al = fr % gamma;
    const int r = r0 + fr / gamma;
    const int sample = (int)blockIdx.z;
    const uint32_t row = fdiv(w, div_Lh);
    const int i = (int)(w - row * div_Lh.d);
    const uint32_t zw_u = fdiv(row, div_L);
    const int y = (int)(row - zw_u * div_L.d);
    const int zw = (int)zw_u;
    const int L = g.L, Lh = g.Lh, nzw = g.L / 32;
    const int d0 = al % 6, dd = (P == q) ? d0 : (d0 + 3) % 6;
    const uint32_t M = ((P + y) & 1) ? 0x55555555u : 0xAAAAAAAAu;  // bits whose site has x offset 1
    uint32_t *pl = planes + ((int64_t)sample * R + r) * np * WP;
#pragma unroll
    for (int bit = 0; bit < 2; ++bit) {
        const uint32_t *Sx = pl + (int64_t)(2 + ((src * gamma + al) * 2 + bit) * 2 + (1 - P)) * WP;
        uint32_t out;
        switch (dd) {
            case 0: out = (Sx[w] & ~M) | (Sx[w - i + (i + 1 == Lh ? 0 : i + 1)] & M); break;
            case 3: out = (Sx[w - i + (i == 0 ? Lh - 1 : i - 1)] & ~M) | (Sx[w] & M); break;
            case 1: out = Sx[((int64_t)zw * L + (y + 1 == L ? 0 : y + 1)) * Lh + i]; break;
            case 4: out = Sx[((int64_t)zw * L + (y == 0 ? L - 1 : y - 1)) * Lh + i]; break;
            case 2: out = __funnelshift_r(Sx[w], Sx[((int64_t)(zw + 1 == nzw ? 0 : zw + 1) * L + y) * Lh + i], 1); break;
            default: out = __funnelshift_l(Sx[((int64_t)(zw == 0 ? nzw - 1 : zw - 1) * L + y) * Lh + i], Sx[w], 1); break;
        }
        pl[(int64_t)(2 + ((dst * gamma + al) * 2 + bit) * 2 + P) * WP + w] = out;
    }
}

__global__ void msg_convert_bonds_kernel(uint32_t *bplanes, const uint8_t *bonds, Geometry g, int64_t S, int64_t WP) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= S * 2 * WP) return;
    const int64_t smp = tid / (2 * WP);
    const int64_t rem = tid - smp * 2 * WP;
    const int p = (int)(rem / WP);
    const int64_t w = rem - (int64_t)p * WP;
    // rows of g.P words; the words from g.Lh on hold no site (zero bond planes)
    const int i = (int)(w % g.P);
    const int y = (int)((w / g.P) % g.L);
    const int zw = (int)(w / ((int64_t)g.P * g.L));
    const int64_t base = (smp * 2 + p) * g.half + ((int64_t)32 * zw * g.L + y) * g.P + i;
    const int64_t zstep = (int64_t)g.L * g.P;
    const int nb = i >= g.Lh ? 0 : (g.L - 32 * zw < 32 ? g.L - 32 * zw : 32);  // sites of the column in this word
    uint32_t bk[6] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nb; ++b) {
        const uint32_t v = bonds[base + b * zstep];
#pragma unroll
        for (int k = 0; k < 6; ++k) bk[k] |= ((v >> k) & 1u) << b;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) bplanes[((smp * 6 + k) * 2 + p) * WP + w] = bk[k];
}

bool msg_supported(const Geometry &g) { return g.L >= 32 && g.L % 32 == 0 && g.P == g.Lh; }

// Words of one plane: L * ceil(L / 32) z words per row of P columns, the byte
// layout's row pitch (Lh rounded up to whole Philox blocks of four; L^3 / 64
// when L is a multiple of 32).
int64_t msg_plane_words(const Geometry &g) { return (int64_t)g.L * ((g.L + 31) / 32) * g.P; }

int msg_planes_per_replica(int gamma, int walkers) { return 2 + 4 * gamma * (walkers ? 2 : 1); }

cudaError_t msg_convert(uint32_t *planes, uint32_t *bplanes, int8_t *spins, uint8_t *daemons, const uint8_t *bonds,
                        const Geometry &g, int S, int R, int gamma, int walkers, int buf, bool to_planes,
                        cudaStream_t st) {
    const int64_t WP = msg_plane_words(g);
    const int64_t n = (int64_t)S * R * 2 * WP;
    msg_convert_state_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        planes, spins, daemons, g, (int64_t)S * R, WP, gamma, msg_planes_per_replica(gamma, walkers), buf, to_planes);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !to_planes || !bplanes) return e;
    return msg_convert_bonds(bplanes, bonds, g, S, st);
}

cudaError_t msg_convert_bonds(uint32_t *bplanes, const uint8_t *bonds, const Geometry &g, int S, cudaStream_t st) {
    const int64_t WP = msg_plane_words(g);
    const int64_t nb = (int64_t)S * 2 * WP;
    msg_convert_bonds_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(bplanes, bonds, g, S, WP);
    return cudaGetLastError();
}

int msg_default_rpt(const Geometry &g, int S, int R, int nw, int sm_count) {  // grid.y = ceil(R / rpt)
    // enough replica groups to fill the GPU (about 2048 threads per SM), the
    // rest of the replicas looped over inside a thread
    const int64_t threads = (int64_t)S * g.L * (g.L / 32) * (g.Lh / nw);
    const int64_t want = (int64_t)sm_count * 2048;
    int groups = (int)std::min<int64_t>(R, std::max<int64_t>(1, (want + threads - 1) / threads));
    return (R + groups - 1) / groups;
}

cudaError_t launch_msg_wander(uint32_t *planes, const Geometry &g, int S, int R, int r0, int r1, int gamma,
                              const SweepParam *params, const int64_t *cursor, int64_t k, bool pdl, cudaStream_t st) {
    const int64_t WP = msg_plane_words(g);
    if (S > 65535 || (int64_t)(r1 - r0) * gamma * 2 > 65535) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((WP + 255) / 256), (unsigned)((r1 - r0) * gamma * 2), (unsigned)S);
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, msg_wander_kernel, planes, g, R, r0, gamma, msg_planes_per_replica(gamma, 1),
                              (uint32_t)WP, make_fastdiv((uint32_t)g.Lh), make_fastdiv((uint32_t)g.L), params, cursor,
                              k);
}

cudaError_t launch_msg_half(uint32_t *planes, const uint32_t *bplanes, const Geometry &g, int S, int R, int r0,
                            int r1, int rpt, int nw, bool regcap, int parity, int gamma, int walkers, uint32_t key0,
                            uint32_t key1, const SweepParam *params, const int64_t *cursor, int64_t k, bool pdl,
                            cudaStream_t st, bool metro) {
    MsgArgs a{};
    a.gamma = gamma;
    a.walkers = walkers;
    a.np = msg_planes_per_replica(gamma, walkers);
    a.planes = planes;
    a.bonds = bplanes;
    a.L = g.L;
    a.Lh = g.Lh;
    a.nzw = g.L / 32;
    a.W4 = g.Lh / 4;
    a.WP = msg_plane_words(g);
    a.S = S;
    a.R = R;
    a.r0 = r0;
    a.r1 = r1;
    a.rpt = rpt;
    a.parity = parity;
    a.key0 = key0;
    a.key1 = key1;
    a.params = params;
    a.cursor = cursor;
    a.k = k;
    a.div_groups = make_fastdiv((uint32_t)(g.Lh / nw));
    a.div_L = make_fastdiv((uint32_t)g.L);
    const int64_t per_sample = (int64_t)g.L * (g.L / 32) * (g.Lh / nw);
    if (per_sample % 128 != 0 || per_sample >= (1ll << 31) || S > 65535 || rpt < 1 || r0 < 0 || r1 > R || r0 >= r1)
        return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(per_sample / 128), (unsigned)((r1 - r0 + rpt - 1) / rpt), (unsigned)S);
    cfg.blockDim = dim3(128);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (metro) {  // Metropolis sweeps on the planes (gamma 1, no walkers)
        if (nw == 4) return cudaLaunchKernelEx(&cfg, msg_half_kernel<4, 4, true>, a);
        if (nw == 2) return cudaLaunchKernelEx(&cfg, msg_half_kernel<2, 4, true>, a);
        return cudaLaunchKernelEx(&cfg, msg_half_kernel<1, 4, true>, a);
    }
    switch (nw * (regcap ? -1 : 1)) {
        case 1: return cudaLaunchKernelEx(&cfg, msg_half_kernel<1, 4>, a);
        case 2: return cudaLaunchKernelEx(&cfg, msg_half_kernel<2, 4>, a);
        case 4: return cudaLaunchKernelEx(&cfg, msg_half_kernel<4, 4>, a);
        case -1: return cudaLaunchKernelEx(&cfg, msg_half_kernel<1, 5>, a);
        case -2: return cudaLaunchKernelEx(&cfg, msg_half_kernel<2, 5>, a);
        case -4: return cudaLaunchKernelEx(&cfg, msg_half_kernel<4, 5>, a);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace micsa
