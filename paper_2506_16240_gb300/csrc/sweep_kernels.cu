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
#include "sweep_body.cuh"

namespace micsa {

__device__ __forceinline__ void grid_dependency_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The grid-stride loops over samples, replicas and chunks for one kind of
// sweep (REF: refresh drawn in the sweep; t and the cut points are used by the
// refresh and Metropolis copies only).
template <int NW, bool METRO, bool FULL, bool REF>
__device__ __forceinline__ void half_sweep_loops(const SweepArgs &a, int alpha, int64_t t, uint64_t th0,
                                                 uint64_t th1, uint64_t th2) {
    const Geometry g = a.geo;
    const uint32_t per_sample = (uint32_t)g.L * g.L * (g.W / NW);  // < 2^31 for L <= 1600
    // grid: x over the chunks of one sample, y over samples; thread row y of
    // the block takes replicas r0 + threadIdx.y, r0 + threadIdx.y + blockDim.y, ... < r1
    for (int sample = blockIdx.y; sample < a.S; sample += gridDim.y)
        for (int r = a.r0 + threadIdx.y; r < a.r1; r += blockDim.y) {
            const int64_t gid = (int64_t)sample * a.R + r;
            // daemon family alpha of this replica; its Philox id is gid * gamma + alpha
            // (Metropolis draws use gid itself)
            const int64_t fam = gid * a.gamma + alpha;
            int8_t *spins = a.spins + gid * 2 * g.half;
            uint8_t *daemons = a.daemons + fam * 2 * g.half;
            const uint8_t *bonds = a.bonds + (int64_t)sample * 2 * g.half;
            for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < per_sample; q += gridDim.x * blockDim.x) {
                const uint32_t row = fdiv(q, a.div_chunks);
                const int c = (int)(q - row * a.div_chunks.d);
                update_chunk<NW, METRO, false, FULL>(g, spins, daemons, bonds, a.parity, (int)row, c,
                                                     (uint32_t)(METRO ? gid : fam), a.key0, a.key1, t, REF, th0,
                                                     th1, th2, a.div_L);
            }
        }
}

template <int NW, bool METRO, bool FULL>
__device__ __forceinline__ void half_sweep_body(const SweepArgs &a) {
    // The sweep's parameters are read before waiting for the previous grid: no
    // kernel of a graph replay writes the table or the replay cursor (the
    // cursor is advanced by the replay's last node, and replays are ordered by
    // the stream), so the dependent loads overlap the wait. Only what selects
    // the copy and the daemon family is read there (every field read there is a
    // load on every sweep's path); a refresh sweep reads its index and cut
    // points in its own copy, Metropolis needs them on every sweep.
    const int64_t kidx = a.k + (a.cursor ? *a.cursor : 0);
    const SweepParam *pp = a.params + kidx;
    const int mode = pp->mode, alpha = pp->alpha;
    int64_t t = 0;
    uint64_t th0 = 0, th1 = 0, th2 = 0;
    if constexpr (METRO) {
        t = pp->t;
        th0 = pp->th0;
        th1 = pp->th1;
        th2 = pp->th2;
    }
    grid_dependency_wait();  // the previous half-sweep's writes are visible after this
    grid_launch_dependents();
    if (METRO) half_sweep_loops<NW, true, FULL, false>(a, 0, t, th0, th1, th2);
    else if (mode == kModeRefresh) half_sweep_loops<NW, false, FULL, true>(a, alpha, pp->t, pp->th0, pp->th1, pp->th2);
    else half_sweep_loops<NW, false, FULL, false>(a, alpha, 0, 0, 0, 0);
}

// One chunk per thread: the grid covers every (chunk, sample, replica) exactly
// once (x: the chunks of a sample, y: samples, z: groups of blockDim.y
// replicas), so the body runs without the loops of half_sweep_body; refresh and
// plain sweeps take separate copies of the update under a branch that is
// uniform over the grid, so neither carries the other's code.
template <int NW, bool METRO, bool FULL>
__device__ __forceinline__ void half_sweep_flat_body(const SweepArgs &a) {
    const int64_t kidx = a.k + (a.cursor ? *a.cursor : 0);
    const SweepParam *pp = a.params + kidx;
    // Only what selects the copy and the daemon family is read before the wait:
    // every field read there is a load on every sweep's path. The sweep index
    // and cut points of a refresh sweep are read in its own copy (a tenth of the
    // sweeps or fewer); Metropolis needs them on every sweep.
    const int mode = pp->mode, alpha = pp->alpha;
    int64_t t = 0;
    uint64_t th0 = 0, th1 = 0, th2 = 0;
    if constexpr (METRO) {
        t = pp->t;
        th0 = pp->th0;
        th1 = pp->th1;
        th2 = pp->th2;
    }
    grid_dependency_wait();
    grid_launch_dependents();
    const Geometry g = a.geo;
    const uint32_t per_sample = (uint32_t)g.L * g.L * (g.W / NW);
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = a.r0 + (int)(blockIdx.z * blockDim.y + threadIdx.y);
    if (q >= per_sample || r >= a.r1) return;
    const uint32_t row = fdiv(q, a.div_chunks);
    const int c = (int)(q - row * a.div_chunks.d);
    const int64_t gid = (int64_t)blockIdx.y * a.R + r;
    const int64_t fam = gid * a.gamma + alpha;
    int8_t *spins = a.spins + gid * 2 * g.half;
    uint8_t *daemons = a.daemons + fam * 2 * g.half;
    const uint8_t *bonds = a.bonds + (int64_t)blockIdx.y * 2 * g.half;
    if (METRO)
        update_chunk<NW, true, false, FULL>(g, spins, daemons, bonds, a.parity, (int)row, c, (uint32_t)gid, a.key0,
                                            a.key1, t, false, th0, th1, th2, a.div_L);
    else if (mode == kModeRefresh)
        update_chunk<NW, false, false, FULL>(g, spins, daemons, bonds, a.parity, (int)row, c, (uint32_t)fam, a.key0,
                                             a.key1, pp->t, true, pp->th0, pp->th1, pp->th2, a.div_L);
    else  // a plain sweep uses neither the sweep index nor cut points
        update_chunk<NW, false, false, FULL>(g, spins, daemons, bonds, a.parity, (int)row, c, (uint32_t)fam, a.key0,
                                             a.key1, 0, false, 0, 0, 0, a.div_L);
}

// FULL: rows without padding (P == L / 2), see update_chunk. FLAT: one chunk
// per thread (half_sweep_flat_body), else the grid-stride loops of
// half_sweep_body (any grid).
template <int NW, bool METRO, bool FULL = false, bool FLAT = false>
__global__ void __launch_bounds__(256) half_sweep_kernel(SweepArgs a) {
    if constexpr (FLAT) half_sweep_flat_body<NW, METRO, FULL>(a);
    else half_sweep_body<NW, METRO, FULL>(a);
}

// The same kernel with registers capped at 64 per thread (8 blocks of 128
// threads per SM): more warps in flight for the latency-bound L2-resident case.
template <int NW, bool METRO, bool FULL = false, bool FLAT = false>
__global__ void __launch_bounds__(128, 8) half_sweep_kernel_rc(SweepArgs a) {
    if constexpr (FLAT) half_sweep_flat_body<NW, METRO, FULL>(a);
    else half_sweep_body<NW, METRO, FULL>(a);
}

// Two rows per thread (rows without padding, MicSA): thread q of a sample takes
// the row pair (z, 2j), (z, 2j + 1) and chunk c, q = (z L/2 + j) chunks + c.
template <int NW>
__global__ void __launch_bounds__(256) half_sweep_pair_kernel(SweepArgs a) {
    const int64_t kidx = a.k + (a.cursor ? *a.cursor : 0);
    const SweepParam prm = a.params[kidx];
    grid_dependency_wait();
    grid_launch_dependents();
    const Geometry g = a.geo;
    const uint32_t per_sample = (uint32_t)g.L * (g.L / 2) * (g.W / NW);
    const bool refresh = prm.mode == kModeRefresh;
    for (int sample = blockIdx.y; sample < a.S; sample += gridDim.y)
        for (int r = a.r0 + threadIdx.y; r < a.r1; r += blockDim.y)
            for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < per_sample; q += gridDim.x * blockDim.x) {
                const uint32_t prow = fdiv(q, a.div_chunks);
                const int c = (int)(q - prow * a.div_chunks.d);
                const uint32_t z = fdiv(prow, a.div_half_L);
                const int y0 = 2 * (int)(prow - z * a.div_half_L.d);
                const int64_t gid = (int64_t)sample * a.R + r;
                const int64_t fam = gid * a.gamma + prm.alpha;
                update_pair<NW>(g, a.spins + gid * 2 * g.half, a.daemons + fam * 2 * g.half,
                                a.bonds + (int64_t)sample * 2 * g.half, a.parity, (int)z, y0, c, (uint32_t)fam,
                                a.key0, a.key1, prm.t, refresh, prm.th0, prm.th1, prm.th2);
            }
}

// All replicas of a sample in one thread (rows without padding, MicSA): thread
// q of a sample takes chunk q of the half-lattice for the replicas [r0, r1),
// loading the bond words and computing the row's offsets once for all of them.
template <int NW>
__global__ void __launch_bounds__(256) half_sweep_reps_kernel(SweepArgs a) {
    const int64_t kidx = a.k + (a.cursor ? *a.cursor : 0);
    const SweepParam prm = a.params[kidx];
    grid_dependency_wait();
    grid_launch_dependents();
    const Geometry g = a.geo;
    const uint32_t per_sample = (uint32_t)g.L * g.L * (g.W / NW);
    const bool refresh = prm.mode == kModeRefresh;
    const int nrep = a.r1 - a.r0;
    for (int sample = blockIdx.y; sample < a.S; sample += gridDim.y)
        for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < per_sample; q += gridDim.x * blockDim.x) {
            const uint32_t row = fdiv(q, a.div_chunks);
            const int c = (int)(q - row * a.div_chunks.d);
            const int64_t gid0 = (int64_t)sample * a.R + a.r0;
            const int64_t fam0 = gid0 * a.gamma + prm.alpha;  // daemon family of the sweep, replica r0
            update_reps<NW>(g, a.spins + gid0 * 2 * g.half, a.daemons + fam0 * 2 * g.half, 2 * g.half,
                            (int64_t)a.gamma * 2 * g.half, a.bonds + (int64_t)sample * 2 * g.half, a.parity,
                            (int)row, c, nrep, (uint32_t)fam0, (uint32_t)a.gamma, a.key0, a.key1, prm.t, refresh,
                            prm.th0, prm.th1, prm.th2, a.div_L);
        }
}

// Wandering (Sec. 2.6): every site of parity p exchanges the walker of family
// alpha with its neighbour along direction alpha mod 6 (+x, +y, +z, -x, -y, -z,
// the table of Sec. 2.8). One thread per (replica family, site of parity p);
// each exchange pair belongs to exactly one thread, and the bytes are moved
// one by one, so no two threads touch the same byte.
__global__ void wander_kernel(uint8_t *daemons, Geometry g, int64_t n_fam, int gamma, int p) {
    const int64_t per = (int64_t)g.L * g.L * g.Lh;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= per * n_fam) return;
    const int64_t fam = tid / per;
    const int64_t rem = tid - fam * per;
    const int row = (int)(rem / g.Lh), i = (int)(rem - (int64_t)row * g.Lh);
    const int y = row % g.L, z = row / g.L;
    const int o = (p + y + z) & 1;
    const int dir = (int)(fam % gamma) % 6;
    int yn = y, zn = z, in = i;
    switch (dir) {
        case 0: in = o ? (i + 1 == g.Lh ? 0 : i + 1) : i; break;   // +x
        case 1: yn = (y + 1 == g.L) ? 0 : y + 1; break;            // +y
        case 2: zn = (z + 1 == g.L) ? 0 : z + 1; break;            // +z
        case 3: in = o ? i : (i == 0 ? g.Lh - 1 : i - 1); break;   // -x
        case 4: yn = (y == 0) ? g.L - 1 : y - 1; break;            // -y
        default: zn = (z == 0) ? g.L - 1 : z - 1; break;           // -z
    }
    uint8_t *own = daemons + (fam * 2 + p) * g.half + (int64_t)row * g.P + i;
    uint8_t *nb = daemons + (fam * 2 + (1 - p)) * g.half + ((int64_t)zn * g.L + yn) * g.P + in;
    const uint8_t a = *own, b = *nb;
    *own = b;
    *nb = a;
}

cudaError_t launch_wander(uint8_t *daemons, Geometry g, int64_t n_rep, int gamma, int parity, cudaStream_t st) {
    const int64_t n = (int64_t)g.L * g.L * g.Lh * n_rep * gamma;
    wander_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(daemons, g, n_rep * gamma, gamma, parity);
    return cudaGetLastError();
}

// Advance the graph replay cursor by `step` sweeps (the last node of a graph).
__global__ void advance_cursor_kernel(int64_t *cursor, int64_t step) {
    grid_dependency_wait();
    grid_launch_dependents();
    *cursor += step;
}

// Block = (chunks per block) x (replica rows, at most 8); `block` is the
// requested total thread count, the chunk dimension a multiple of 32, and the
// block never exceeds max_threads (the kernel's launch bound: 128 for the
// register-capped kernels, 256 for the others).
dim3 block_shape(int R, int block, int max_threads) {
    int ry = R < 8 ? R : 8;
    if (ry > max_threads / 32) ry = max_threads / 32;
    int cx = block / ry;
    cx = cx < 32 ? 32 : (cx / 32) * 32;
    while (cx > 32 && cx * ry > max_threads) cx -= 32;
    return dim3((unsigned)cx, (unsigned)ry);
}

template <int NW, bool METRO>
static cudaError_t launch_variant(const SweepArgs &a0, const LaunchConfig &lc, cudaStream_t st) {
    SweepArgs a = a0;
    const int chunks = a.geo.W / NW;
    a.div_chunks = make_fastdiv((uint32_t)chunks);
    a.div_L = make_fastdiv((uint32_t)a.geo.L);
    const int64_t per_sample = (int64_t)a.geo.L * a.geo.L * chunks;
    const dim3 blk = block_shape(a.r1 - a.r0, lc.regcap && lc.block > 128 ? 128 : lc.block, lc.regcap ? 128 : 256);
    int64_t gx = (per_sample + blk.x - 1) / blk.x;
    int64_t gy = a.S < 65535 ? a.S : 65535;
    // no grid cap and every sample on its own grid row: one chunk per thread
    const bool flat = lc.max_blocks <= 0 && a.S <= 65535;
    const int64_t gz = flat ? (a.r1 - a.r0 + blk.y - 1) / blk.y : 1;
    if (lc.max_blocks > 0 && gx * gy > lc.max_blocks) {  // grid-stride cap over chunks
        gx = lc.max_blocks / gy > 0 ? lc.max_blocks / gy : 1;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)gx, (unsigned)gy, (unsigned)gz);
    cfg.blockDim = blk;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = lc.pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const bool full = a.geo.P == a.geo.Lh;
    if (flat) {
        if (lc.regcap)
            return full ? cudaLaunchKernelEx(&cfg, half_sweep_kernel_rc<NW, METRO, true, true>, a)
                        : cudaLaunchKernelEx(&cfg, half_sweep_kernel_rc<NW, METRO, false, true>, a);
        return full ? cudaLaunchKernelEx(&cfg, half_sweep_kernel<NW, METRO, true, true>, a)
                    : cudaLaunchKernelEx(&cfg, half_sweep_kernel<NW, METRO, false, true>, a);
    }
    if (lc.regcap)
        return full ? cudaLaunchKernelEx(&cfg, half_sweep_kernel_rc<NW, METRO, true>, a)
                    : cudaLaunchKernelEx(&cfg, half_sweep_kernel_rc<NW, METRO, false>, a);
    return full ? cudaLaunchKernelEx(&cfg, half_sweep_kernel<NW, METRO, true>, a)
                : cudaLaunchKernelEx(&cfg, half_sweep_kernel<NW, METRO, false>, a);
}

int vector_words(const Geometry &g, int want) {
    if (want >= 4 && g.W % 4 == 0) return 4;
    if (want >= 2 && g.W % 2 == 0) return 2;
    return 1;
}

template <int NW>
static cudaError_t launch_pairs(const SweepArgs &a0, const LaunchConfig &lc, cudaStream_t st) {
    SweepArgs a = a0;
    const int chunks = a.geo.W / NW;
    a.div_chunks = make_fastdiv((uint32_t)chunks);
    a.div_half_L = make_fastdiv((uint32_t)(a.geo.L / 2));
    const int64_t per_sample = (int64_t)a.geo.L * (a.geo.L / 2) * chunks;
    const dim3 blk = block_shape(a.r1 - a.r0, lc.block, 256);
    int64_t gx = (per_sample + blk.x - 1) / blk.x;
    int64_t gy = a.S < 65535 ? a.S : 65535;
    if (lc.max_blocks > 0 && gx * gy > lc.max_blocks) gx = lc.max_blocks / gy > 0 ? lc.max_blocks / gy : 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)gx, (unsigned)gy);
    cfg.blockDim = blk;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = lc.pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, half_sweep_pair_kernel<NW>, a);
}

template <int NW>
static cudaError_t launch_reps(const SweepArgs &a0, const LaunchConfig &lc, cudaStream_t st) {
    SweepArgs a = a0;
    const int chunks = a.geo.W / NW;
    a.div_chunks = make_fastdiv((uint32_t)chunks);
    a.div_L = make_fastdiv((uint32_t)a.geo.L);
    const int64_t per_sample = (int64_t)a.geo.L * a.geo.L * chunks;
    const int blk = lc.block;
    int64_t gx = (per_sample + blk - 1) / blk;
    int64_t gy = a.S < 65535 ? a.S : 65535;
    if (lc.max_blocks > 0 && gx * gy > lc.max_blocks) gx = lc.max_blocks / gy > 0 ? lc.max_blocks / gy : 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)gx, (unsigned)gy);
    cfg.blockDim = dim3((unsigned)blk);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = lc.pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, half_sweep_reps_kernel<NW>, a);
}

// Row pairs apply to MicSA half-sweeps of rows without padding.
bool pairs_apply(const Geometry &g, bool metro, const LaunchConfig &lc) {
    return lc.pairs && !metro && g.P == g.Lh && g.L % 2 == 0;
}

// Replicas in one thread apply to MicSA half-sweeps of rows without padding.
bool reps_apply(const Geometry &g, bool metro, const LaunchConfig &lc) {
    return lc.reps && !lc.pairs && !metro && g.P == g.Lh;
}

cudaError_t launch_half_sweep(const SweepArgs &a, bool metro, const LaunchConfig &lc, cudaStream_t st) {
    const int nw = vector_words(a.geo, lc.nw);
    if (reps_apply(a.geo, metro, lc))
        return nw == 4 ? launch_reps<4>(a, lc, st) : nw == 2 ? launch_reps<2>(a, lc, st) : launch_reps<1>(a, lc, st);
    if (pairs_apply(a.geo, metro, lc))
        return nw == 4 ? launch_pairs<4>(a, lc, st) : nw == 2 ? launch_pairs<2>(a, lc, st) : launch_pairs<1>(a, lc, st);
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

template <int NW, bool METRO>
static int occupancy(bool rc, int block) {
    int n = 0;
    const cudaError_t e = rc ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, half_sweep_kernel_rc<NW, METRO>, block, 0)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, half_sweep_kernel<NW, METRO>, block, 0);
    return e == cudaSuccess ? n : 0;
}

int max_resident_blocks_pairs(int nw, int block) {
    int n = 0;
    const cudaError_t e =
        nw == 4 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, half_sweep_pair_kernel<4>, block, 0)
        : nw == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, half_sweep_pair_kernel<2>, block, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, half_sweep_pair_kernel<1>, block, 0);
    return e == cudaSuccess ? n : 0;
}

int max_resident_blocks_reps(int nw, int block) {
    int n = 0;
    const cudaError_t e =
        nw == 4 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, half_sweep_reps_kernel<4>, block, 0)
        : nw == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, half_sweep_reps_kernel<2>, block, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, half_sweep_reps_kernel<1>, block, 0);
    return e == cudaSuccess ? n : 0;
}

int max_resident_blocks(bool metro, int nw, int block, bool regcap) {
    if (metro) return nw == 4 ? occupancy<4, true>(regcap, block) : nw == 2 ? occupancy<2, true>(regcap, block)
                                                                   : occupancy<1, true>(regcap, block);
    return nw == 4 ? occupancy<4, false>(regcap, block) : nw == 2 ? occupancy<2, false>(regcap, block)
                                                        : occupancy<1, false>(regcap, block);
}

}  // namespace micsa
