// sweep_kernels.cu -- the hot loop: one checkerboard half-sweep of MicSA
// (Sec. 2.8 procedure steps (i)/(ii)) with the daemon refresh of Sec. 2.7
// fused in, and the same-layout Metropolis half-sweep used as the
// random-number-greedy comparison (Sec. 2.3, App. B).
//
// One thread owns NW consecutive 32-bit words (4 NW sites) of one row of the
// own parity and updates them for every replica of its sample, so the bond
// bytes and the neighbour addressing are shared by the R replicas. Per word and
// replica it reads the own spin and daemon words and the five opposite-parity
// neighbour words (same row, y +- 1, z +- 1) and writes the spin and daemon
// words back. On a refresh sweep the daemon word is drawn, not read.
//
// The per-sweep parameters (t, cut points, refresh or not) come from a device
// table so that one captured CUDA graph of G sweeps can be replayed for a
// whole run; consecutive half-sweeps are chained with programmatic dependent
// launch (griddepcontrol) so that a grid is scheduled while its predecessor
// drains.
#include "micsa_internal.h"

namespace micsa {

__device__ __forceinline__ void grid_dependency_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <int NW, bool METRO>
__global__ void __launch_bounds__(256) half_sweep_kernel(SweepArgs a) {
    grid_dependency_wait();  // the previous half-sweep's writes are visible after this
    grid_launch_dependents();
    const Geometry g = a.geo;
    const int chunks = g.W / NW;
    const int64_t per_sample = (int64_t)g.L * g.L * chunks;
    const int64_t total = per_sample * a.S;
    const int64_t kidx = a.k + (a.cursor ? *a.cursor : 0);
    const SweepParam prm = a.params[kidx];
    const bool refresh = !METRO && prm.mode == kModeRefresh;
    const int p = a.parity;

    // thread row y of the block takes replicas y, y + blockDim.y, ...
    for (int r = threadIdx.y; r < a.R; r += blockDim.y)
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int sample = (int)(q / per_sample);
        const int64_t rem = q - (int64_t)sample * per_sample;
        const int row = (int)(rem / chunks);
        const int c = (int)(rem - (int64_t)row * chunks);
        const int y = row % g.L, z = row / g.L;
        const int o = (p + y + z) & 1;
        const int b0 = c * 4 * NW;  // first byte of this thread's range within the row

        const int yp = (y + 1 == g.L) ? 0 : y + 1, ym = (y == 0) ? g.L - 1 : y - 1;
        const int zp = (z + 1 == g.L) ? 0 : z + 1, zm = (z == 0) ? g.L - 1 : z - 1;
        const int64_t row0 = (int64_t)row * g.P;
        const int64_t off_c = row0 + b0;
        const int64_t gid = (int64_t)sample * a.R + r;
        const int8_t *__restrict__ opp = a.spins + (gid * 2 + (1 - p)) * g.half;
        int8_t *__restrict__ own_s = a.spins + (gid * 2 + p) * g.half;
        uint8_t *__restrict__ own_d = a.daemons + (gid * 2 + p) * g.half;

        uint32_t Bw[NW], O[NW], Oyp[NW], Oym[NW], Ozp[NW], Ozm[NW], S[NW], D[NW];
        load_words_ro<NW>(a.bonds + (int64_t)(sample * 2 + p) * g.half + off_c, Bw);
        load_words_ro<NW>(opp + off_c, O);
        load_words_ro<NW>(opp + ((int64_t)z * g.L + yp) * g.P + b0, Oyp);
        load_words_ro<NW>(opp + ((int64_t)z * g.L + ym) * g.P + b0, Oym);
        load_words_ro<NW>(opp + ((int64_t)zp * g.L + y) * g.P + b0, Ozp);
        load_words_ro<NW>(opp + ((int64_t)zm * g.L + y) * g.P + b0, Ozm);
        load_words<NW>(own_s + off_c, S);
        if (!METRO && !refresh) load_words<NW>(own_d + off_c, D);

        // edge bytes for the x shift and the periodic wrap of the row
        uint32_t edge = 0, first = 0, last = 0;
        if (o == 0) {
            if (b0 == 0) last = (uint8_t)__ldg(opp + row0 + g.Lh - 1);
            else edge = (uint8_t)__ldg(opp + off_c - 1);
        } else {
            if (b0 + 4 * NW <= g.Lh - 1) edge = (uint8_t)__ldg(opp + off_c + 4 * NW);
            else first = (b0 == 0) ? (O[0] & 0xFFu) : (uint8_t)__ldg(opp + row0);
        }
        uint32_t xp[NW], xm[NW];
        x_neighbours<NW>(O, o, b0, g.Lh, edge, first, last, xp, xm);
        const uint32_t quad0 = (uint32_t)((((int64_t)p * g.L + z) * g.L + y) * g.W + c * NW);

#pragma unroll
        for (int j = 0; j < NW; ++j) {
            const BondPlanes bp = bond_planes(Bw[j]);
            const uint32_t neg = negative_terms(bp, xp[j], xm[j], Oyp[j], Oym[j], Ozp[j], Ozm[j]);
            const uint32_t u32 = unsatisfied32(neg, S[j]);
            const uint32_t valid = valid_mask(b0, j, g.Lh);
            if (METRO) {
                // dH = 12 - 4u > 0 <=> u < 3; accept iff a fresh uniform is below
                // the Metropolis cut point of dH (index 2 - u).
                const uint4 w = philox4x32_10(
                    make_uint4(quad0 + j, (uint32_t)prm.t, (uint32_t)(gid << 2) | kTagMetro,
                               (uint32_t)((uint64_t)prm.t >> 32)),
                    a.key0, a.key1);
                uint32_t am = 0;
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    const uint32_t u = (u32 >> (8 * l + 5)) & 7u;
                    bool acc = u >= 3;
                    if (!acc) {
                        const uint64_t cut = (u == 2) ? prm.th0 : (u == 1) ? prm.th1 : prm.th2;
                        acc = (uint64_t)lane_of(w, l) < cut;
                    }
                    if (acc) am |= 0xFFu << (8 * l);
                }
                am &= valid;
                S[j] ^= am & 0xFEFEFEFEu;
            } else {
                if (refresh) {
                    const uint4 w = philox4x32_10(
                        make_uint4(quad0 + j, (uint32_t)prm.t, (uint32_t)(gid << 2) | kTagDaemon,
                                   (uint32_t)((uint64_t)prm.t >> 32)),
                        a.key0, a.key1);
                    D[j] = daemon_from_uniform(w.x, prm.th0, prm.th1, prm.th2) |
                           (daemon_from_uniform(w.y, prm.th0, prm.th1, prm.th2) << 8) |
                           (daemon_from_uniform(w.z, prm.th0, prm.th1, prm.th2) << 16) |
                           (daemon_from_uniform(w.w, prm.th0, prm.th1, prm.th2) << 24);
                    D[j] &= valid;
                }
                const uint32_t am = creutz4(u32, D[j], valid);
                S[j] ^= am & 0xFEFEFEFEu;
            }
        }
        store_words<NW>(own_s + off_c, S);
        if (!METRO) store_words<NW>(own_d + off_c, D);
    }
}

// Advance the graph replay cursor by `step` sweeps (the last node of a graph).
__global__ void advance_cursor_kernel(int64_t *cursor, int64_t step) {
    grid_dependency_wait();
    grid_launch_dependents();
    *cursor += step;
}

// Block = (chunks per block) x (replica rows, at most 8); `block` is the
// requested total thread count, the chunk dimension a multiple of 32.
dim3 block_shape(int R, int block) {
    const int ry = R < 8 ? R : 8;
    int cx = block / ry;
    cx = cx < 32 ? 32 : (cx / 32) * 32;
    while (cx > 32 && cx * ry > 256) cx -= 32;
    return dim3((unsigned)cx, (unsigned)ry);
}

template <int NW, bool METRO>
static cudaError_t launch_variant(const SweepArgs &a, const LaunchConfig &lc, cudaStream_t st) {
    const int64_t chunks = (int64_t)a.S * a.geo.L * a.geo.L * (a.geo.W / NW);
    const dim3 blk = block_shape(a.R, lc.block);
    int64_t grid = (chunks + blk.x - 1) / blk.x;
    if (lc.max_blocks > 0 && grid > lc.max_blocks) grid = lc.max_blocks;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = blk;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = lc.pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, half_sweep_kernel<NW, METRO>, a);
}

int vector_words(const Geometry &g, int want) {
    if (want >= 4 && g.W % 4 == 0) return 4;
    if (want >= 2 && g.W % 2 == 0) return 2;
    return 1;
}

cudaError_t launch_half_sweep(const SweepArgs &a, bool metro, const LaunchConfig &lc, cudaStream_t st) {
    const int nw = vector_words(a.geo, lc.nw);
    if (metro) {
        if (nw == 4) return launch_variant<4, true>(a, lc, st);
        if (nw == 2) return launch_variant<2, true>(a, lc, st);
        return launch_variant<1, true>(a, lc, st);
    }
    if (nw == 4) return launch_variant<4, false>(a, lc, st);
    if (nw == 2) return launch_variant<2, false>(a, lc, st);
    return launch_variant<1, false>(a, lc, st);
}

cudaError_t launch_advance_cursor(int64_t *cursor, int64_t step, bool pdl, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(1);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, advance_cursor_kernel, cursor, step);
}

int max_resident_blocks(bool metro, int nw, int block) {
    int n = 0;
    cudaError_t e;
    if (metro)
        e = nw == 4 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, half_sweep_kernel<4, true>, block, 0)
          : nw == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, half_sweep_kernel<2, true>, block, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, half_sweep_kernel<1, true>, block, 0);
    else
        e = nw == 4 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, half_sweep_kernel<4, false>, block, 0)
          : nw == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, half_sweep_kernel<2, false>, block, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, half_sweep_kernel<1, false>, block, 0);
    return e == cudaSuccess ? n : 0;
}

}  // namespace micsa
