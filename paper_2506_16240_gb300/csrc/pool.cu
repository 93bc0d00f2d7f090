// pool.cu -- the batched engine: many independent annealing jobs of mixed L,
// replicas, sweep counts and refresh intervals resident in one device arena,
// advanced together by one persistent grid-stride launch per half-sweep, a tick
// of K sweeps replayed as one CUDA graph. Jobs are admitted and retired between
// ticks (continuous batching): admission is limited by free slots and by free
// arena memory.
//
// A job is micsa_create(L, 1, R, seed) + micsa_run with the linear schedule
// T(k) = T_start + (T_end - T_start) * (k / (n_sweeps - 1)) and its refresh
// interval: the same Philox counters (sample 0, gid = replica), so its result
// does not depend on which slot it occupies or on which jobs run beside it.
// After every tick each job's exact energy is measured and the lowest energy
// seen so far (ties: the earliest) is kept together with that configuration.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include <cooperative_groups.h>

#include "sweep_body.cuh"
#include "msg_body.cuh"
#include "../../include/micsa.h"

namespace micsa {

constexpr int kPoolMaxR = MICSA_POOL_MAX_REPLICAS;
constexpr int kVBlock = 128;  // chunk items per virtual block
constexpr int kPoolMaxChains = 4;  // parts of the streaming jobs run as concurrent kernel chains (default 2)



struct VBlock {
    int32_t slot;
    int16_t replica;
    int16_t pad;
    int32_t chunk0;  // first chunk of the replica's half-lattice in this block
};

// 128 threads of one bit-plane job: thread q updates (and converts) the plane
// words 4q .. 4q + 3 of every replica, q = chunk0 + threadIdx.x.
struct PVBlock {
    int32_t slot;
    int32_t chunk0;
};

// One unit of the shared-memory bit-plane kernel: replicas [r0, r0 + nrep) of
// the bit-plane job in `slot`, held in one CTA's shared memory for a tick;
// bonds_smem: the job's bond planes are copied there too (else read from the
// arena, where they stay in L2).
struct PlaneUnit {
    int32_t slot;
    int16_t r0, nrep;
    int16_t bonds_smem;
    int16_t C;  // 1: the unit in one CTA; C > 1: a cluster of C CTAs, CTA c holding z word c
};

constexpr int kMaxCluster = 4;  // clusters of 2..4 CTAs: L up to 128

// CTA sizes of the shared-memory bit-plane kernel: 512 threads for one CTA per
// SM, 256 threads for two or more (registers: about 120 per thread)
constexpr int kSmemPlaneThreads = 512;
constexpr int kSmemPlaneThreadsSmall = 256;
// lattices with L <= 32: units of a few replicas in CTAs of 128 threads, four per SM
constexpr int kSmallPlaneThreads = 128;
constexpr int kSmallPlaneBlocks = 4;
constexpr size_t kSmallPlaneSmem = 48 << 10;

struct PoolTables {
    JobDesc *jobs;          // [max_jobs]
    const VBlock *vblocks;  // [max_vblocks]
    const int32_t *n_vblocks;  // [kPoolMaxChains + 1]: the end of each chain's part over the byte-streamed
                               // jobs (unused parts: their total); [kPoolMaxChains]: all the jobs measured
                               // over the table (byte-streamed first, then the bit-plane jobs)
    const PVBlock *pvblocks;   // the bit-plane jobs' half-sweep blocks
    const int32_t *n_pvb;      // [kPoolMaxChains]: the end of each chain's part (unused parts: the total)
    long long *energy;      // [max_jobs][kPoolMaxR]
    long long *aux;
    long long *best_energy;
    long long *best_t;
    unsigned long long *acc;  // [max_jobs][kPoolMaxR][2] energy and daemon sums of the tick (zero between ticks)
    int32_t *improved;        // [max_jobs][kPoolMaxR] the tick's energy is the lowest so far
};

__device__ __forceinline__ void pool_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pool_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// The job-level values of one half-sweep of a job, read from its descriptor
// once per run of virtual blocks of that job.
struct PoolJobState {
    Geometry geo;
    int8_t *spins;
    uint8_t *daemons;
    const uint8_t *bonds;
    int64_t t;
    uint32_t c0m, c1m, c2m;  // refresh cut points minus one (each in [2^30, 2^32])
    uint32_t key0, key1, chunks;
    FastDiv dc, divL;
    int nw;
    bool active, refresh, full;
};

__device__ __forceinline__ void load_job_state(const JobDesc &J, int k, PoolJobState &s) {
    s.t = J.t + k;
    s.active = J.live && s.t < J.n_sweeps;
    s.geo = J.geo;
    s.spins = J.spins;
    s.daemons = J.daemons;
    s.bonds = J.bonds;
    s.key0 = J.key0;
    s.key1 = J.key1;
    s.nw = J.nw;
    s.full = s.geo.P == s.geo.Lh;  // rows without padding
    s.chunks = (uint32_t)s.geo.L * s.geo.L * (s.geo.W / s.nw);
    s.dc = FastDiv{(uint32_t)(s.geo.W / s.nw), J.divC_m, J.divC_l};
    s.divL = FastDiv{(uint32_t)s.geo.L, J.divL_m, J.divL_l};
    s.refresh = s.active && (s.t % J.interval) == 0;
    s.c0m = s.c1m = s.c2m = 0;
    if (s.refresh) {
        const uint64_t *q = J.thr + 3 * (s.t / J.interval);
        s.c0m = (uint32_t)(q[0] - 1);
        s.c1m = (uint32_t)(q[1] - 1);
        s.c2m = (uint32_t)(q[2] - 1);
    }
}

template <int NW, bool FULL>
__device__ __forceinline__ void pool_item(const PoolJobState &s, int r, uint32_t chunk, int p) {
    const uint32_t row = fdiv(chunk, s.dc);
    const int c = (int)(chunk - row * s.dc.d);
    const int64_t roff = (int64_t)r * 2 * s.geo.half;
    update_chunk<NW, false, false, FULL>(s.geo, s.spins + roff, s.daemons + roff, s.bonds, p, (int)row, c,
                                         (uint32_t)r, s.key0, s.key1, s.t, s.refresh, (uint64_t)s.c0m + 1,
                                         (uint64_t)s.c1m + 1, (uint64_t)s.c2m + 1, s.divL);
}

// One half-sweep (parity p) of sweep k of the tick for every live job of part
// `part` of the virtual-block table (the parts hold disjoint (job, replica)
// pairs and run as concurrent kernel chains).
__global__ void __launch_bounds__(kVBlock, 5) pool_half_sweep_kernel(PoolTables T, int k, int p, int part) {
    pool_wait();
    pool_release();
    const int v0 = part == 0 ? 0 : T.n_vblocks[part - 1];
    const int nvb = T.n_vblocks[part] - v0;
    // a contiguous run of virtual blocks per CTA: mostly one job (its state is
    // read once per run) and neighbouring planes (their rows are re-read from L1)
    const int per = (nvb + (int)gridDim.x - 1) / (int)gridDim.x;
    const int vb_end = v0 + min(nvb, ((int)blockIdx.x + 1) * per);
    PoolJobState s;
    int slot = -1;  // the job whose state s holds (the same for every thread of the CTA)
    for (int vb = v0 + (int)blockIdx.x * per; vb < vb_end; ++vb) {
        const VBlock b = T.vblocks[vb];
        if (b.slot != slot) {
            slot = b.slot;
            load_job_state(T.jobs[slot], k, s);
        }
        if (!s.active) continue;
        const uint32_t chunk = (uint32_t)b.chunk0 + threadIdx.x;
        if (chunk >= s.chunks) continue;
        if (s.nw == 4) s.full ? pool_item<4, true>(s, b.replica, chunk, p) : pool_item<4, false>(s, b.replica, chunk, p);
        else if (s.nw == 2) s.full ? pool_item<2, true>(s, b.replica, chunk, p) : pool_item<2, false>(s, b.replica, chunk, p);
        else s.full ? pool_item<1, true>(s, b.replica, chunk, p) : pool_item<1, false>(s, b.replica, chunk, p);
    }
}

// Energy of the even sites and daemon energy of NW words of one chunk of row
// (z, y) of one replica: H_EA = sum over even sites of (2u - 6), every bond
// having exactly one even end for even L; H_aux = 4 * sum of m over both
// parities. Same neighbour assembly as update_chunk.
template <int NW, bool FULL>
__device__ __forceinline__ void chunk_measure(const Geometry &g, const int8_t *sp, const uint8_t *dm,
                                              const uint8_t *bonds, int row, int c, const FastDiv &divL, int &e,
                                              int &a) {
    const int z = (int)fdiv((uint32_t)row, divL), y = row - z * g.L;
    const int o = (y + z) & 1;
    const int b0 = c * 4 * NW;
    const int yp = (y + 1 == g.L) ? 0 : y + 1, ym = (y == 0) ? g.L - 1 : y - 1;
    const int zp = (z + 1 == g.L) ? 0 : z + 1, zm = (z == 0) ? g.L - 1 : z - 1;
    const int64_t row0 = (int64_t)row * g.P, off = row0 + b0;
    const int8_t *odd = sp + g.half;
    uint32_t O[NW], Oyp[NW], Oym[NW], Ozp[NW], Ozm[NW], B[NW], S[NW], D0[NW], D1[NW];
    load_words<NW>(odd + off, O);
    load_words<NW>(odd + ((int64_t)z * g.L + yp) * g.P + b0, Oyp);
    load_words<NW>(odd + ((int64_t)z * g.L + ym) * g.P + b0, Oym);
    load_words<NW>(odd + ((int64_t)zp * g.L + y) * g.P + b0, Ozp);
    load_words<NW>(odd + ((int64_t)zm * g.L + y) * g.P + b0, Ozm);
    load_words<NW>(bonds + off, B);
    load_words<NW>(sp + off, S);
    load_words<NW>(dm + off, D0);
    load_words<NW>(dm + g.half + off, D1);
    uint32_t edge = 0, first = 0, last = 0;
    if constexpr (FULL) {
        const int8_t *ep = o == 0 ? (b0 == 0 ? odd + row0 + g.Lh - 1 : odd + off - 1)
                                  : (b0 + 4 * NW < g.Lh ? odd + off + 4 * NW : odd + row0);
        edge = last = (uint8_t)*ep;
    } else if (o == 0) {
        if (b0 == 0) last = (uint8_t)odd[row0 + g.Lh - 1];
        else edge = (uint8_t)odd[off - 1];
    } else {
        if (b0 + 4 * NW <= g.Lh - 1) edge = (uint8_t)odd[off + 4 * NW];
        else first = (b0 == 0) ? (O[0] & 0xFFu) : (uint8_t)odd[row0];
    }
    uint32_t xp[NW], xm[NW];
    x_neighbours<NW, !FULL>(O, o, b0, g.Lh, edge, first, last, xp, xm);
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        const uint32_t valid = FULL ? 0xFFFFFFFFu : valid_mask(b0, j, g.Lh);
        const uint32_t u32 =
            unsatisfied_count(B[j], S[j], xp[j], xm[j], Oyp[j], Oym[j], Ozp[j], Ozm[j]) & valid;
        e += 2 * (int)(((u32 >> 5) * 0x01010101u) >> 24) - 6 * (__popc(valid) / 8);
        a += 4 * (int)((((D0[j] & valid) * 0x01010101u) >> 24) + (((D1[j] & valid) * 0x01010101u) >> 24));
    }
}

// Bit-plane jobs, at the start and at the end of a tick: their byte state
// to planes (to_planes) or back, each thread the 4 words of its half-sweep
// position, both parities, every replica.
__global__ void __launch_bounds__(kVBlock) pool_planes_convert_kernel(PoolTables T, int to_planes, int part) {
    pool_wait();
    pool_release();
    const int v0 = part == 0 ? 0 : T.n_pvb[part - 1];
    const int nvb = T.n_pvb[part] - v0;
    const int per = (nvb + (int)gridDim.x - 1) / (int)gridDim.x;
    const int vb_end = v0 + min(nvb, ((int)blockIdx.x + 1) * per);
    for (int vb = v0 + (int)blockIdx.x * per; vb < vb_end; ++vb) {
        const PVBlock b = T.pvblocks[vb];
        const JobDesc &J = T.jobs[b.slot];
        if (!J.live || J.t >= J.n_sweeps) continue;
        const Geometry g = J.geo;
        const int64_t WP = (int64_t)g.L * ((g.L + 31) / 32) * g.P;
        const int64_t w0 = 4 * ((int64_t)b.chunk0 + threadIdx.x);
        if (w0 >= WP) continue;
        for (int r = 0; r < J.R; ++r)
            for (int par = 0; par < 2; ++par)
                for (int j = 0; j < 4; ++j)
                    msg_convert_word(J.planes, J.spins, J.daemons, g, WP, 1, 6, 0, to_planes != 0, r, par, w0 + j);
    }
}

// One half-sweep (parity p) of sweep k of the tick for every live bit-plane
// job: the bit-plane update of the single-handle engine with ragged z columns
// (4 words per thread,
// every replica of the job in one thread, the job's own clock, cut points and
// Philox key; replica r is Philox id r, as in the byte path).
__global__ void __launch_bounds__(kVBlock, 4) pool_msg_half_kernel(PoolTables T, int k, int p, int part) {
    pool_wait();
    pool_release();
    const int v0 = part == 0 ? 0 : T.n_pvb[part - 1];
    const int nvb = T.n_pvb[part] - v0;
    const int per = (nvb + (int)gridDim.x - 1) / (int)gridDim.x;
    const int vb_end = v0 + min(nvb, ((int)blockIdx.x + 1) * per);
    int slot = -1;  // the job whose state is held below (the same for the whole CTA)
    MsgLattice lat{};
    SweepParam prm{};
    FastDiv dg{}, dL{};
    int R = 0;
    bool active = false;
    for (int vb = v0 + (int)blockIdx.x * per; vb < vb_end; ++vb) {
        const PVBlock b = T.pvblocks[vb];
        if (b.slot != slot) {
            slot = b.slot;
            const JobDesc &J = T.jobs[slot];
            const int64_t t = J.t + k;
            active = J.live && t < J.n_sweeps;
            const Geometry g = J.geo;
            const int nzw = (g.L + 31) / 32;
            lat = MsgLattice{J.planes, J.bplanes, g.L, g.P, nzw, g.P / 4, (int64_t)g.L * nzw * g.P,
                             6, 1, 0, 0, J.key0, J.key1, g.Lh};
            prm = SweepParam{};
            prm.t = t;
            prm.mode = kModeMicsa;
            if (active && t % J.interval == 0) {
                const uint64_t *q = J.thr + 3 * (t / J.interval);
                prm.th0 = q[0];
                prm.th1 = q[1];
                prm.th2 = q[2];
                prm.mode = kModeRefresh;
            }
            dg = make_fastdiv_dev((uint32_t)(g.P / 4));
            dL = make_fastdiv_dev((uint32_t)g.L);
            R = J.R;
        }
        if (!active) continue;
        const uint32_t q = (uint32_t)b.chunk0 + threadIdx.x;
        if ((int64_t)q * 4 >= lat.WP) continue;  // (job thread counts are multiples of 128)
        const uint32_t rowi = fdiv(q, dg);
        const uint32_t zw = fdiv(rowi, dL);
        msg_update<4, true, false, true, true>(lat, prm, p, (int)zw, (int)(rowi - zw * dL.d), (int)(q - rowi * dg.d), 0, R);
    }
}

// ------------------------------------------ bit-plane jobs in shared memory --
// Dynamic shared memory of pool_smem_planes_kernel: the unit's planes
// [replica][spin p0, p1, m0 p0, p1, m1 p0, p1][WP], then (when held here) the
// bond planes [direction][parity][WP].
extern __shared__ __align__(16) uint32_t pool_spl[];

// One unit's geometry as the shared-memory update sees it: rows of P plane words
// (Lr of them sites), nzw z words per column (Lz sites in the last), W4 = P / 4
// Philox blocks per row.
struct SplaneGeo {
    int L, P, Lr, nzw, W4, Lz;
    uint32_t WP;
    FastDiv dW4, dL;
    uint32_t bonds_off;  // word offset of the bond planes in shared memory
    uint32_t bwp;        // words between consecutive bond planes (shared memory or global)
    // a cluster's CTA: the z word it holds and the shared memory of the CTAs
    // holding the next and the previous z word (generic addresses)
    int zw0;
    const uint32_t *up, *dn;
};

__device__ __forceinline__ void lds4(uint32_t idx, uint32_t (&v)[4]) {
    const uint4 a = *reinterpret_cast<const uint4 *>(&pool_spl[idx]);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
}

__device__ __forceinline__ void sts4(uint32_t idx, const uint32_t (&v)[4]) {
    *reinterpret_cast<uint4 *>(&pool_spl[idx]) = make_uint4(v[0], v[1], v[2], v[3]);
}

// Half-sweep (parity p) of word group q (the plane words i0 .. i0 + 3 of one
// (zw, y) row, i0 = 4 (q mod W4)) for replicas [0, nrep) of the unit held in
// shared memory: the same move as the global bit-plane update (Eq. (Creutz)
// with Eq. (flip-OK), bit-sliced; at a refresh sweep the daemons of the words
// are drawn first from the same Philox blocks, Sec. 2.7), with 32-bit shared
// memory indices. BSMEM: the bond planes are in shared memory, else at gb.
// CL: the CTA holds one z word (G.zw0) of a unit split over a cluster; the
// opposite-parity words at z word zw0 +- 1 are read from the CTAs holding them
// (distributed shared memory), at the same index within their slice.
template <bool BSMEM, bool CL = false>
__device__ __forceinline__ void splane_group(const SplaneGeo &G, const uint32_t *gb, int p, uint32_t q, int nrep,
                                             int64_t t, bool refresh, const CutsGt &cut, const RoundKeys &rk,
                                             uint32_t gid0) {
    const uint32_t rowi = fdiv(q, G.dW4);
    const uint32_t zw = CL ? 0u : fdiv(rowi, G.dL);  // z word within this CTA's planes
    const uint32_t zwg = CL ? (uint32_t)G.zw0 : zw;   // the z word in the lattice
    const int L = G.L;
    const int y = (int)(rowi - zw * (uint32_t)L);
    const int i0 = 4 * (int)(q - rowi * (uint32_t)G.W4);
    const int o = 1 - p;
    const int yp = (y + 1 == L) ? 0 : y + 1, ym = (y == 0) ? L - 1 : y - 1;
    const uint32_t zwp = (zw + 1 == (uint32_t)G.nzw) ? 0u : zw + 1, zwm = (zw == 0) ? (uint32_t)G.nzw - 1 : zw - 1;
    const int ip = (i0 + 4 >= G.Lr) ? 0 : i0 + 4, im = (i0 == 0) ? G.Lr - 1 : i0 - 1;
    const uint32_t P = (uint32_t)G.P, row = zw * (uint32_t)L;
    const uint32_t wc = (row + y) * P + i0;
    const uint32_t w_yp = (row + yp) * P + i0, w_ym = (row + ym) * P + i0;
    const uint32_t w_zp = CL ? wc : (zwp * L + y) * P + i0, w_zm = CL ? wc : (zwm * L + y) * P + i0;
    const uint32_t w_ip = (row + y) * P + ip, w_im = (row + y) * P + im;
    const uint32_t M = ((p + y) & 1) ? 0x55555555u : 0xAAAAAAAAu;  // bits whose site has x offset 1
    const bool zlast = zwg + 1 == (uint32_t)G.nzw, zfirst = zwg == 0;
    const int Lz = G.Lz;
    const uint32_t zmask = (zlast && Lz < 32) ? ((1u << Lz) - 1u) : 0xFFFFFFFFu;
    uint32_t wmask[4];  // words from Lr on are padding: no site
#pragma unroll
    for (int w = 0; w < 4; ++w) wmask[w] = i0 + w < G.Lr ? zmask : 0u;

    uint32_t B[6][4];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const uint32_t bi = (uint32_t)(k * 2 + p) * G.bwp + wc;
        if constexpr (BSMEM) {
            lds4(G.bonds_off + bi, B[k]);
        } else {
            const uint4 a = __ldg(reinterpret_cast<const uint4 *>(gb + bi));
            B[k][0] = a.x;
            B[k][1] = a.y;
            B[k][2] = a.z;
            B[k][3] = a.w;
        }
    }
    const uint32_t quad0 = (((uint32_t)p * L + 32 * zwg) * L + y) * (uint32_t)G.W4 + (uint32_t)(i0 >> 2);
    for (int r = 0; r < nrep; ++r) {
        const uint32_t base = (uint32_t)r * 6 * G.WP;
        const uint32_t Ob = base + (uint32_t)o * G.WP, Sb = base + (uint32_t)p * G.WP;
        const uint32_t M0b = base + (uint32_t)(2 + p) * G.WP, M1b = base + (uint32_t)(4 + p) * G.WP;
        uint32_t Oc[4], Oyp[4], Oym[4], Ozp[4], Ozm[4], Sg[4], m0v[4], m1v[4];
        lds4(Ob + wc, Oc);
        lds4(Ob + w_yp, Oyp);
        lds4(Ob + w_ym, Oym);
        if constexpr (CL) {
            const uint4 a = *reinterpret_cast<const uint4 *>(G.up + Ob + w_zp);
            const uint4 b = *reinterpret_cast<const uint4 *>(G.dn + Ob + w_zm);
            Ozp[0] = a.x; Ozp[1] = a.y; Ozp[2] = a.z; Ozp[3] = a.w;
            Ozm[0] = b.x; Ozm[1] = b.y; Ozm[2] = b.z; Ozm[3] = b.w;
        } else {
            lds4(Ob + w_zp, Ozp);
            lds4(Ob + w_zm, Ozm);
        }
        const uint32_t Oip = pool_spl[Ob + w_ip], Oim = pool_spl[Ob + w_im];
        lds4(Sb + wc, Sg);
        if (refresh) {
            // fresh daemons of parity p (Sec. 2.7): the Philox block of z = 32 zw + b
            // holds the uniforms of the four words; bits enter from the top z down
            uint32_t x0[4] = {0, 0, 0, 0}, x1[4] = {0, 0, 0, 0}, x2[4] = {0, 0, 0, 0};
            const uint32_t n0 = ~cut.c0m, n1 = ~cut.c1m, n2 = ~cut.c2m;
            const uint32_t fam = gid0 + (uint32_t)r;
#pragma unroll 2
            for (int b = 31; b >= 0; --b) {
                const uint4 u = philox_wide(make_uint4(quad0 + (uint32_t)b * (uint32_t)L * (uint32_t)G.W4, (uint32_t)t,
                                                       (fam << 2) | kTagDaemon, (uint32_t)((uint64_t)t >> 32)),
                                            rk);
                shift_in_cuts(u.x, n0, n1, n2, x0[0], x1[0], x2[0]);
                shift_in_cuts(u.y, n0, n1, n2, x0[1], x1[1], x2[1]);
                shift_in_cuts(u.z, n0, n1, n2, x0[2], x1[2], x2[2]);
                shift_in_cuts(u.w, n0, n1, n2, x0[3], x1[3], x2[3]);
            }
#pragma unroll
            for (int w = 0; w < 4; ++w) {  // m = [u >= c0] + [u >= c1] + [u >= c2]: m1 = x1, m0 = the parity
                m0v[w] = (x0[w] ^ x1[w] ^ x2[w]) & wmask[w];
                m1v[w] = x1[w] & wmask[w];
            }
        } else {
            lds4(M0b + wc, m0v);
            lds4(M1b + wc, m1v);
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const uint32_t oc = Oc[w];
            const uint32_t o_next = (w + 1 < 4 && i0 + w + 1 < G.Lr) ? Oc[w + 1 < 4 ? w + 1 : 0] : Oip;
            const uint32_t o_prev = w > 0 ? Oc[w > 0 ? w - 1 : 0] : Oim;
            const uint32_t nxp = (oc & ~M) | (o_next & M);
            const uint32_t nxm = (o_prev & ~M) | (oc & M);
            const uint32_t nzp = zlast ? (oc >> 1) | ((Ozp[w] & 1u) << (Lz - 1)) : __funnelshift_r(oc, Ozp[w], 1);
            const uint32_t nzm = zfirst ? (oc << 1) | ((Ozm[w] >> (Lz - 1)) & 1u) : __funnelshift_l(Ozm[w], oc, 1);
            const uint32_t sg = Sg[w];
            // unsatisfied bond indicators (J s s_nb = -1), their count u, v = u + m
            const uint32_t q0 = sg ^ nxp ^ B[0][w];
            const uint32_t q1 = sg ^ Oyp[w] ^ B[1][w];
            const uint32_t q2 = sg ^ nzp ^ B[2][w];
            const uint32_t q3 = sg ^ nxm ^ B[3][w];
            const uint32_t q4 = sg ^ Oym[w] ^ B[4][w];
            const uint32_t q5 = sg ^ nzm ^ B[5][w];
            const uint32_t s1 = q0 ^ q1 ^ q2, c1 = (q0 & q1) | (q2 & (q0 ^ q1));
            const uint32_t s2 = q3 ^ q4 ^ q5, c2 = (q3 & q4) | (q5 & (q3 ^ q4));
            const uint32_t u0 = s1 ^ s2, kk = s1 & s2;
            const uint32_t u1 = c1 ^ c2 ^ kk, u2 = (c1 & c2) | (kk & (c1 ^ c2));
            const uint32_t m0 = m0v[w], m1 = m1v[w];
            const uint32_t v0 = u0 ^ m0, k0 = u0 & m0;
            const uint32_t v1 = u1 ^ m1 ^ k0, k1 = (u1 & m1) | (k0 & (u1 ^ m1));
            const uint32_t v2 = u2 ^ k1, v3 = u2 & k1;
            // Eq. (Creutz) with Eq. (flip-OK): accept <=> 3 <= u + m <= 6, m' = u + m - 3
            const uint32_t acc = (v2 ^ (v1 & v0)) & ~v3 & wmask[w];
            m0v[w] = (m0 & ~acc) | (~v0 & acc);
            m1v[w] = (m1 & ~acc) | (v2 & (v1 | v0) & acc);
            Sg[w] = sg ^ acc;
        }
        sts4(Sb + wc, Sg);
        sts4(M0b + wc, m0v);
        sts4(M1b + wc, m1v);
    }
}

// The tick of the bit-plane jobs whose state fits in shared memory: a
// persistent kernel whose CTAs take units (a job's replica range) from a work
// counter, convert the replicas' bytes to bit planes in shared memory (the
// layout of the global bit planes: [replica][spin p0, p1, m0 p0, p1, m1 p0, p1][WP]),
// run the job's K sweeps of this tick there -- the even half-sweep, then the
// odd one, each the body of the global bit-plane kernel (msg_update) over the
// CTA's word groups, the refresh at the job's refresh sweeps -- and convert
// back. No state leaves the SM between the half-sweeps of a tick.
// IDX: the unit table's part and work counter: 1 for the units of L > 32 held in
// one CTA, 0 for the small lattices (L <= 32; counter kMaxCluster + 1).
template <int NT, int MINB, int IDX = 1>
__global__ void __launch_bounds__(NT, MINB)
    pool_smem_planes_kernel(PoolTables T, const PlaneUnit *units, const int32_t *unit_start,
                            const int32_t *n_units, int *counters, int K) {
    pool_wait();
    pool_release();
    uint32_t *spl = pool_spl;
    __shared__ int s_unit;
    const int n = n_units[IDX];
    units += unit_start[IDX];  // the units held in one CTA
    int *counter = counters + (IDX == 0 ? kMaxCluster + 1 : IDX);
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1);
        __syncthreads();
        const int u = s_unit;
        __syncthreads();  // every thread has read s_unit before thread 0 writes the next one
        if (u >= n) break;
        const PlaneUnit U = units[u];
        const JobDesc &J = T.jobs[U.slot];
        if (!J.live || J.t >= J.n_sweeps) continue;
        const Geometry g = J.geo;
        const int nzw = (g.L + 31) / 32;
        const int64_t WP = (int64_t)g.L * nzw * g.P;  // rows of P words (padded to whole Philox blocks)
        const int nrep = U.nrep;
        int8_t *spins = J.spins + (int64_t)U.r0 * 2 * g.half;
        uint8_t *daemons = J.daemons + (int64_t)U.r0 * 2 * g.half;
        uint32_t *sb = spl + (int64_t)nrep * 6 * WP;  // bond planes, when they are held here
        for (int64_t idx = threadIdx.x; idx < (int64_t)nrep * 2 * WP; idx += blockDim.x) {
            const int rep = (int)(idx / (2 * WP));
            const int64_t rem = idx - (int64_t)rep * 2 * WP;
            const int par = (int)(rem / WP);
            msg_convert_word(spl, spins, daemons, g, WP, 1, 6, 0, true, rep, par, rem - par * WP);
        }
        if (U.bonds_smem) {
            const uint4 *src = reinterpret_cast<const uint4 *>(J.bplanes);
            uint4 *dst = reinterpret_cast<uint4 *>(sb);
            for (int64_t i = threadIdx.x; i < 3 * WP; i += blockDim.x) dst[i] = src[i];  // 12 WP words
        }
        __syncthreads();
        SplaneGeo G;
        G.L = g.L;
        G.P = g.P;
        G.Lr = g.Lh;
        G.nzw = nzw;
        G.W4 = g.P / 4;
        G.Lz = g.L - 32 * (nzw - 1);
        G.WP = (uint32_t)WP;
        G.dW4 = make_fastdiv_dev((uint32_t)G.W4);
        G.dL = make_fastdiv_dev((uint32_t)g.L);
        G.bonds_off = (uint32_t)(nrep * 6 * WP);
        G.bwp = (uint32_t)WP;
        G.zw0 = 0;
        G.up = G.dn = nullptr;
        const RoundKeys rk = round_keys(J.key0, J.key1);
        const uint32_t groups = (uint32_t)(WP / 4);
        // a thread's word groups: ceil(groups / threads) each, spread over as many
        // threads as that needs, so that no pass runs with a few threads only
        const uint32_t per = (groups + blockDim.x - 1) / blockDim.x;
        const uint32_t span = (groups + per - 1) / per;  // threads in use
        for (int k = 0; k < K; ++k) {
            const int64_t t = J.t + k;
            if (t >= J.n_sweeps) break;
            const bool refresh = t % J.interval == 0;
            CutsGt cut{0, 0, 0};
            if (refresh) {
                const uint64_t *th = J.thr + 3 * (t / J.interval);
                cut = make_cuts_gt(th[0], th[1], th[2]);
            }
            for (int par = 0; par < 2; ++par) {
                if (threadIdx.x < span)
                    for (uint32_t q = threadIdx.x; q < groups; q += span) {
                        if (U.bonds_smem)
                            splane_group<true>(G, nullptr, par, q, nrep, t, refresh, cut, rk, (uint32_t)U.r0);
                        else
                            splane_group<false>(G, J.bplanes, par, q, nrep, t, refresh, cut, rk, (uint32_t)U.r0);
                    }
                __syncthreads();
            }
        }
        for (int64_t idx = threadIdx.x; idx < (int64_t)nrep * 2 * WP; idx += blockDim.x) {
            const int rep = (int)(idx / (2 * WP));
            const int64_t rem = idx - (int64_t)rep * 2 * WP;
            const int par = (int)(rem / WP);
            msg_convert_word(spl, spins, daemons, g, WP, 1, 6, 0, false, rep, par, rem - par * WP);
        }
        __syncthreads();  // the planes are read out before the next unit overwrites them
    }
}

// Bytes <-> the slice of z word zw0 of one replica's planes in shared memory:
// word w = y P + i of a slice plane holds, in bit b, the site of row (z, y),
// byte i, z = 32 zw0 + b (b < nb); the words from Lh on are padding (zero).
// Slice layout per replica: [spin p0, p1, m0 p0, p1, m1 p0, p1][S].
__device__ __forceinline__ void slice_convert_word(uint32_t *spl, int8_t *spins, uint8_t *daemons, const Geometry &g,
                                                   uint32_t S, int zw0, bool to_planes, int rep, int p, uint32_t w) {
    const int i = (int)(w % (uint32_t)g.P), y = (int)(w / (uint32_t)g.P);
    uint32_t *pl = spl + (uint32_t)rep * 6 * S;
    if (i >= g.Lh) {
        if (to_planes) pl[(uint32_t)p * S + w] = pl[(uint32_t)(2 + p) * S + w] = pl[(uint32_t)(4 + p) * S + w] = 0;
        return;
    }
    const int64_t base = ((int64_t)rep * 2 + p) * g.half + ((int64_t)32 * zw0 * g.L + y) * g.P + i;
    const int64_t zstep = (int64_t)g.L * g.P;
    const int nb = g.L - 32 * zw0 < 32 ? g.L - 32 * zw0 : 32;
    if (to_planes) {
        uint32_t sv = 0, m0 = 0, m1 = 0;
        for (int b = 0; b < nb; ++b) {
            sv |= (((uint32_t)(uint8_t)spins[base + b * zstep] >> 7) & 1u) << b;
            const uint32_t m = daemons[base + b * zstep];
            m0 |= (m & 1u) << b;
            m1 |= ((m >> 1) & 1u) << b;
        }
        pl[(uint32_t)p * S + w] = sv;
        pl[(uint32_t)(2 + p) * S + w] = m0;
        pl[(uint32_t)(4 + p) * S + w] = m1;
    } else {
        const uint32_t sv = pl[(uint32_t)p * S + w], m0 = pl[(uint32_t)(2 + p) * S + w], m1 = pl[(uint32_t)(4 + p) * S + w];
        for (int b = 0; b < nb; ++b) {
            spins[base + b * zstep] = ((sv >> b) & 1u) ? (int8_t)-1 : (int8_t)1;
            daemons[base + b * zstep] = (uint8_t)(((m0 >> b) & 1u) | (((m1 >> b) & 1u) << 1));
        }
    }
}

// The shared-memory bit-plane tick with each unit split over a thread-block
// cluster of C CTAs, CTA c holding z word c of every column of the unit's
// replicas (and of the bond planes when they are held): the z neighbours across
// word boundaries come from the peer CTAs' shared memory, and a cluster barrier
// separates the half-sweeps. Rank 0 takes the units from the work counter and
// the other CTAs read the index from its shared memory.
template <int NT>
__global__ void __launch_bounds__(NT, 1)
    pool_cluster_planes_kernel(PoolTables T, const PlaneUnit *units, const int32_t *unit_start,
                               const int32_t *n_units, int *counters, int K) {
    namespace cg = cooperative_groups;
    pool_wait();
    pool_release();
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), c = (int)cl.block_rank();
    uint32_t *spl = pool_spl;
    __shared__ int s_unit;
    const int n = n_units[C], u0 = unit_start[C];
    int *counter = counters + C;
    const uint32_t *up = cl.map_shared_rank(spl, (c + 1) % C);
    const uint32_t *dn = cl.map_shared_rank(spl, (c + C - 1) % C);
    const int *unit_of_rank0 = cl.map_shared_rank(&s_unit, 0);
    for (;;) {
        if (c == 0 && threadIdx.x == 0) s_unit = atomicAdd(counter, 1);
        cl.sync();
        const int u = *unit_of_rank0;
        cl.sync();  // every CTA has read the index before rank 0 takes the next one
        if (u >= n) break;
        const PlaneUnit U = units[u0 + u];
        const JobDesc &J = T.jobs[U.slot];
        if (!J.live || J.t >= J.n_sweeps) continue;
        const Geometry g = J.geo;
        const int nzw = (g.L + 31) / 32;
        const uint32_t S = (uint32_t)g.L * (uint32_t)g.P;  // words of a slice plane
        const uint32_t WP = (uint32_t)nzw * S;             // words of a global plane
        const int nrep = U.nrep;
        int8_t *spins = J.spins + (int64_t)U.r0 * 2 * g.half;
        uint8_t *daemons = J.daemons + (int64_t)U.r0 * 2 * g.half;
        for (uint32_t idx = threadIdx.x; idx < (uint32_t)nrep * 2 * S; idx += blockDim.x) {
            const int rep = (int)(idx / (2 * S));
            const uint32_t rem = idx - (uint32_t)rep * 2 * S;
            const int par = (int)(rem / S);
            slice_convert_word(spl, spins, daemons, g, S, c, true, rep, par, rem - par * S);
        }
        uint32_t *sb = spl + (uint32_t)nrep * 6 * S;
        if (U.bonds_smem)  // slice c of each of the 12 bond planes
            for (uint32_t i = threadIdx.x; i < 12 * (S / 4); i += blockDim.x) {
                const uint32_t k = i / (S / 4), j = i - k * (S / 4);
                reinterpret_cast<uint4 *>(sb + k * S)[j] =
                    reinterpret_cast<const uint4 *>(J.bplanes + (size_t)k * WP + (size_t)c * S)[j];
            }
        cl.sync();  // every slice is in place before a peer reads it
        SplaneGeo G;
        G.L = g.L;
        G.P = g.P;
        G.Lr = g.Lh;
        G.nzw = nzw;
        G.W4 = g.P / 4;
        G.Lz = g.L - 32 * (nzw - 1);
        G.WP = S;
        G.dW4 = make_fastdiv_dev((uint32_t)G.W4);
        G.dL = make_fastdiv_dev((uint32_t)g.L);
        G.bonds_off = (uint32_t)nrep * 6 * S;
        G.bwp = U.bonds_smem ? S : WP;
        G.zw0 = c;
        G.up = up;
        G.dn = dn;
        const uint32_t *gb = J.bplanes + (size_t)c * S;  // this slice of the global bond planes
        const RoundKeys rk = round_keys(J.key0, J.key1);
        const uint32_t groups = S / 4;
        const uint32_t per = (groups + blockDim.x - 1) / blockDim.x;
        const uint32_t span = (groups + per - 1) / per;
        for (int k = 0; k < K; ++k) {
            const int64_t t = J.t + k;
            if (t >= J.n_sweeps) break;
            const bool refresh = t % J.interval == 0;
            CutsGt cut{0, 0, 0};
            if (refresh) {
                const uint64_t *th = J.thr + 3 * (t / J.interval);
                cut = make_cuts_gt(th[0], th[1], th[2]);
            }
            for (int par = 0; par < 2; ++par) {
                if (threadIdx.x < span)
                    for (uint32_t q = threadIdx.x; q < groups; q += span) {
                        if (U.bonds_smem)
                            splane_group<true, true>(G, nullptr, par, q, nrep, t, refresh, cut, rk, (uint32_t)U.r0);
                        else
                            splane_group<false, true>(G, gb, par, q, nrep, t, refresh, cut, rk, (uint32_t)U.r0);
                    }
                cl.sync();  // the half-sweep's words are visible to the peers
            }
        }
        for (uint32_t idx = threadIdx.x; idx < (uint32_t)nrep * 2 * S; idx += blockDim.x) {
            const int rep = (int)(idx / (2 * S));
            const uint32_t rem = idx - (uint32_t)rep * 2 * S;
            const int par = (int)(rem / S);
            slice_convert_word(spl, spins, daemons, g, S, c, false, rep, par, rem - par * S);
        }
    }
}

// Energy and daemon sums of every (live, advancing) streaming job replica after
// the tick, over the virtual-block table of the half-sweeps: per warp one
// atomic into the (slot, replica) accumulators.
__global__ void __launch_bounds__(kVBlock) pool_energy_kernel(PoolTables T) {
    pool_wait();
    pool_release();
    const int nvb = T.n_vblocks[kPoolMaxChains];
    // a contiguous run of virtual blocks per CTA: mostly one job (its descriptor
    // stays in L1) and neighbouring planes (their rows are re-read from L1)
    const int per = (nvb + (int)gridDim.x - 1) / (int)gridDim.x;
    const int vb_end = min(nvb, ((int)blockIdx.x + 1) * per);
    for (int vb = (int)blockIdx.x * per; vb < vb_end; ++vb) {
        const VBlock b = T.vblocks[vb];
        const JobDesc &J = T.jobs[b.slot];
        if (!J.live || J.t >= J.n_sweeps) continue;
        const Geometry g = J.geo;
        const uint32_t chunks = (uint32_t)g.L * g.L * (g.W / J.nw);
        const uint32_t chunk = (uint32_t)b.chunk0 + threadIdx.x;
        int e = 0, a = 0;
        if (chunk < chunks) {
            const FastDiv dc{(uint32_t)(g.W / J.nw), J.divC_m, J.divC_l};
            const FastDiv divL{(uint32_t)g.L, J.divL_m, J.divL_l};
            const uint32_t row = fdiv(chunk, dc);
            const int c = (int)(chunk - row * dc.d);
            const int8_t *sp = J.spins + (int64_t)b.replica * 2 * g.half;
            const uint8_t *dm = J.daemons + (int64_t)b.replica * 2 * g.half;
            const bool full = g.P == g.Lh;
            if (J.nw == 4) full ? chunk_measure<4, true>(g, sp, dm, J.bonds, (int)row, c, divL, e, a)
                              : chunk_measure<4, false>(g, sp, dm, J.bonds, (int)row, c, divL, e, a);
            else if (J.nw == 2) full ? chunk_measure<2, true>(g, sp, dm, J.bonds, (int)row, c, divL, e, a)
                                     : chunk_measure<2, false>(g, sp, dm, J.bonds, (int)row, c, divL, e, a);
            else full ? chunk_measure<1, true>(g, sp, dm, J.bonds, (int)row, c, divL, e, a)
                      : chunk_measure<1, false>(g, sp, dm, J.bonds, (int)row, c, divL, e, a);
        }
        e = __reduce_add_sync(0xFFFFFFFFu, e);
        a = __reduce_add_sync(0xFFFFFFFFu, a);
        if ((threadIdx.x & 31) == 0) {
            unsigned long long *acc = T.acc + ((size_t)b.slot * kPoolMaxR + b.replica) * 2;
            atomicAdd(acc, (unsigned long long)(long long)e);
            atomicAdd(acc + 1, (unsigned long long)(long long)a);
        }
    }
}

// Results of the tick per (slot, replica): energy, daemon energy, and whether
// the energy is the lowest so far (then also the sweep count); the accumulators
// are cleared for the next tick. One block of 32 threads per slot.
__global__ void pool_best_kernel(PoolTables T, int K) {
    pool_wait();
    pool_release();
    const int slot = blockIdx.x, r = threadIdx.x;
    if (r >= kPoolMaxR) return;
    const JobDesc &J = T.jobs[slot];
    const int cell = slot * kPoolMaxR + r;
    T.improved[cell] = 0;
    if (!J.live || J.resident || r >= J.R || J.t >= J.n_sweeps) return;
    const long long e = (long long)T.acc[2 * cell], a = (long long)T.acc[2 * cell + 1];
    T.acc[2 * cell] = 0;
    T.acc[2 * cell + 1] = 0;
    T.energy[cell] = e;
    T.aux[cell] = a;
    if (e < T.best_energy[cell]) {
        T.best_energy[cell] = e;
        T.best_t[cell] = J.t + K < J.n_sweeps ? J.t + K : J.n_sweeps;
        T.improved[cell] = 1;
    }
}

// Copy of the configurations whose energy improved, in the split layout (the
// natural layout is produced when the job is polled), over the virtual blocks.
__global__ void __launch_bounds__(kVBlock) pool_best_copy_kernel(PoolTables T) {
    pool_wait();
    pool_release();
    const int nvb = T.n_vblocks[kPoolMaxChains];
    // a contiguous run of virtual blocks per CTA: mostly one job (its descriptor
    // stays in L1) and neighbouring planes (their rows are re-read from L1)
    const int per = (nvb + (int)gridDim.x - 1) / (int)gridDim.x;
    const int vb_end = min(nvb, ((int)blockIdx.x + 1) * per);
    for (int vb = (int)blockIdx.x * per; vb < vb_end; ++vb) {
        const VBlock b = T.vblocks[vb];
        if (!T.improved[b.slot * kPoolMaxR + b.replica]) continue;
        const JobDesc &J = T.jobs[b.slot];
        const Geometry g = J.geo;
        const uint32_t chunks = (uint32_t)g.L * g.L * (g.W / J.nw);
        const uint32_t chunk = (uint32_t)b.chunk0 + threadIdx.x;
        if (chunk >= chunks) continue;
        const int64_t off = (int64_t)chunk * 4 * J.nw;  // chunks tile the rows contiguously
        const int8_t *src = J.spins + (int64_t)b.replica * 2 * g.half;
        int8_t *dst = J.best + (int64_t)b.replica * 2 * g.half;
        for (int par = 0; par < 2; ++par)
            for (int w = 0; w < J.nw; ++w)
                *reinterpret_cast<uint32_t *>(dst + par * g.half + off + 4 * w) =
                    *reinterpret_cast<const uint32_t *>(src + par * g.half + off + 4 * w);
    }
}

// t <- min(t + K, n_sweeps) for every live job (the last node of a tick).
__global__ void pool_advance_kernel(JobDesc *jobs, int max_jobs, int K, int *counter) {
    pool_wait();
    pool_release();
    if (blockIdx.x == 0 && threadIdx.x <= kMaxCluster + 1) counter[threadIdx.x] = 0;  // the next tick's persistent kernels' work counters
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max_jobs; i += gridDim.x * blockDim.x) {
        JobDesc &J = jobs[i];
        if (!J.live) continue;
        J.t = J.t + K < J.n_sweeps ? J.t + K : J.n_sweeps;
    }
}

static cudaError_t launch_pdl(const void *fn, dim3 grid, dim3 block, cudaStream_t st, void **args, bool pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace micsa

using namespace micsa;

// ------------------------------------------------------------------ host --
struct PoolJob {
    int64_t id = -1;
    micsa_job_desc desc{};
    size_t off_bonds = 0, off_spins = 0, off_daemons = 0, off_best = 0, off_thr = 0, off_planes = 0, off_bplanes = 0,
           bytes = 0;
    int64_t t = 0;           // host mirror of sweeps done after the queued ticks
    int64_t done_tick = -1;  // tick index whose completion finishes the job
    bool live = false;
};

struct micsa_pool {
    int device = 0, sm_count = 0;
    int max_jobs = 0, K = 64;
    size_t arena_bytes = 0;
    uint8_t *arena = nullptr;
    std::map<size_t, size_t> free_list;  // offset -> size
    JobDesc *d_jobs = nullptr;           // device table
    std::vector<JobDesc> h_jobs;         // host mirror (t follows every queued tick)
    JobDesc *h_jobs_stage = nullptr;     // pinned copy being uploaded
    VBlock *d_vblocks = nullptr, *h_vblocks = nullptr;  // h_vblocks: pinned upload source
    int32_t *d_nvb = nullptr, *h_nvb = nullptr;
    int max_vblocks = 0;
    long long *d_results = nullptr;  // energy | aux | best_energy | best_t, [max_jobs][kPoolMaxR] each
    unsigned long long *d_acc = nullptr;  // per-tick energy / daemon sums of the streaming jobs
    int32_t *d_improved = nullptr;        // per (slot, replica): the last tick improved the best energy
    std::vector<PoolJob> slots;
    int64_t next_id = 1;
    int64_t ticks_queued = 0;
    std::vector<cudaEvent_t> tick_events;  // ring of events, one per queued tick
    int64_t launches = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    cudaStream_t aux_stream = nullptr;       // forked branch of a tick (resident kernel)
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    cudaStream_t chain_stream[kPoolMaxChains] = {};  // forked branches: parts 1.. of the streaming jobs
    cudaEvent_t chain_fork = nullptr, chain_join[kPoolMaxChains] = {};
    int chains = 2;     // concurrent kernel chains over the streaming jobs (1..kPoolMaxChains)
    int max_words = 4;  // words per thread of a streaming job: the largest of 4, 2, 1 <= max_words dividing W
    bool tables_dirty = true;
    cudaEvent_t tables_free = nullptr;  // the last table upload has been consumed
    // per slot: pinned staging of the job's initial data (cut points + result
    // reset values) and the event after which it may be overwritten
    std::vector<uint64_t *> stage;
    std::vector<size_t> stage_cap;
    std::vector<cudaEvent_t> stage_free;
    int grid_blocks = 0;
    bool pdl = true;
    int use_graph = 1;
    // resident (shared-memory) part: jobs whose replica fits kResidentBudget
    size_t resident_smem = 0;  // 0: resident kernel disabled
    int resident_grid = 0;
    ResidentUnit *d_units = nullptr, *h_units = nullptr;  // h_units: pinned upload source
    int32_t *d_nunits = nullptr, *h_nunits = nullptr;
    int *d_counter = nullptr;
    int max_units = 0;
    bool has_stream_jobs = false, has_resident_jobs = false, has_plane_jobs = false;
    // bit-plane jobs (even L above 32): forked branches of the tick
    bool planes_on = true;  // for the jobs admitted from now on
    PVBlock *d_pvblocks = nullptr, *h_pvblocks = nullptr;
    int32_t *d_npvb = nullptr, *h_npvb = nullptr;
    int max_pvblocks = 0;
    int planes_grid = 0;
    cudaStream_t planes_stream[kPoolMaxChains] = {};  // the bit-plane jobs' parts as concurrent chains
    cudaEvent_t planes_fork = nullptr, planes_join[kPoolMaxChains] = {};
    // bit-plane jobs swept in shared memory (one persistent launch per tick)
    size_t splanes_smem = 0;  // per-CTA shared-memory budget for the jobs admitted from now on; 0: off
    size_t splanes_max_smem = 0;  // what the device allows the kernel
    int splanes_grid = 0;
    bool splanes_cluster = true;  // split the units of jobs with L > 32 over clusters (jobs admitted from now on)
    bool small_planes = false;    // jobs with L <= 32 as bit planes in shared memory (else the multispin kernel)
    int small_grid = 0;
    PlaneUnit *d_punits = nullptr, *h_punits = nullptr;
    // per cluster size C (index 1..kMaxCluster): first unit and unit count in the table
    int32_t *d_npunits = nullptr, *h_npunits = nullptr, *d_pustart = nullptr, *h_pustart = nullptr;
    int max_punits = 0;
    size_t splanes_launch_smem[kMaxCluster + 1] = {};  // the largest unit of each cluster size
    int cluster_grid[kMaxCluster + 1] = {};            // CTAs of the launch of each cluster size
    cudaStream_t splanes_stream[kMaxCluster + 2] = {};  // [kMaxCluster + 1]: the small lattices' launch
    cudaEvent_t splanes_fork = nullptr, splanes_join[kMaxCluster + 2] = {};
    cudaGraphExec_t graphs[256] = {};  // by part mask: 1 resident, 2 byte-streamed, 4 bit-plane jobs,
                                       // 8 << (C - 1): bit-plane jobs in shared memory, units over C CTAs,
                                       // 8 << kMaxCluster: the small lattices' units
    std::string err;
};

namespace {

int pfail(micsa_pool_t p, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
int pfail(micsa_pool_t p, int code, const char *fmt, ...) {
    if (p) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        p->err = buf;
    }
    return code;
}

#define PCK(p, expr, what)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return pfail(p, e_ == cudaErrorMemoryAllocation ? MICSA_E_OOM : MICSA_E_CUDA, "%s: %s", \
                         what, cudaGetErrorString(e_));                                      \
    } while (0)

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool arena_alloc(micsa_pool_t p, size_t bytes, size_t *off) {
    bytes = align_up(bytes);
    for (auto it = p->free_list.begin(); it != p->free_list.end(); ++it) {
        if (it->second >= bytes) {
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t new_off = it->first + bytes;
            p->free_list.erase(it);
            if (rest) p->free_list[new_off] = rest;
            return true;
        }
    }
    return false;
}

void arena_free(micsa_pool_t p, size_t off, size_t bytes) {
    bytes = align_up(bytes);
    auto it = p->free_list.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != p->free_list.end() && it->first + it->second == next->first) {
        it->second += next->second;
        p->free_list.erase(next);
    }
    if (it != p->free_list.begin()) {
        auto prev = std::prev(it);
        if (prev->first + prev->second == it->first) {
            prev->second += it->second;
            p->free_list.erase(it);
        }
    }
}

size_t arena_free_bytes(const micsa_pool_t p) {
    size_t s = 0;
    for (auto &kv : p->free_list) s += kv.second;
    return s;
}

double schedule_T(const micsa_job_desc &d, int64_t k) {
    if (d.n_sweeps <= 1) return d.T_start;
    return d.T_start + (d.T_end - d.T_start) * ((double)k / (double)(d.n_sweeps - 1));
}

struct JobSizes {
    Geometry g;
    size_t bonds, state, best, thr, planes, bplanes;  // planes, bplanes: 0 unless plane_eligible
    int64_t n_refresh;
};

// Jobs the bit-plane path can take: every even L above the shared-memory
// multispin kernel's sizes (L > 32): rows of P = 4 ceil(Lh / 4) plane words (whole
// Philox blocks; the words from Lh on are padding), z columns in 32-bit words,
// the last one partial when L is not a multiple of 32.
bool plane_eligible(const micsa_job_desc &d) { return d.L % 2 == 0 && d.L > 32; }

// Units of a bit-plane job in the shared-memory kernel for a per-CTA budget of
// `smem` bytes: all replicas with the bond planes when they fit, else as many
// replicas as fit beside the bond planes, else replicas without them; nrep = 0
// if one replica's six planes do not fit.
struct SplaneSplit {
    int nrep;
    bool bonds_smem;
    size_t bytes;  // shared memory of one unit
};

SplaneSplit splane_split(int64_t WP, int R, size_t smem) {
    const size_t wb = sizeof(uint32_t) * (size_t)WP;  // one plane
    if (!smem) return {0, false, 0};
    if ((6 * (size_t)R + 12) * wb <= smem) return {R, true, (6 * (size_t)R + 12) * wb};
    if (18 * wb <= smem) {
        const int n = (int)std::min<size_t>((size_t)R, (smem / wb - 12) / 6);
        return {n, true, (6 * (size_t)n + 12) * wb};
    }
    if (6 * wb <= smem) {
        const int n = (int)std::min<size_t>((size_t)R, smem / (6 * wb));
        return {n, false, 6 * (size_t)n * wb};
    }
    return {0, false, 0};
}

JobSizes job_sizes(const micsa_job_desc &d) {
    JobSizes s;
    s.g = make_geometry(d.L);
    s.bonds = (size_t)2 * s.g.half;
    s.state = (size_t)d.n_replicas * 2 * s.g.half;
    // natural layout (shared-memory jobs) or the split layout (streaming jobs)
    s.best = (size_t)d.n_replicas * std::max<size_t>((size_t)d.L * d.L * d.L, (size_t)2 * s.g.half);
    s.n_refresh = (d.n_sweeps + d.refresh_interval - 1) / d.refresh_interval;
    if (s.n_refresh < 1) s.n_refresh = 1;
    s.thr = sizeof(uint64_t) * 3 * (size_t)s.n_refresh;
    const size_t WP = (size_t)msg_plane_words(s.g);
    s.planes = plane_eligible(d) ? sizeof(uint32_t) * 6 * WP * (size_t)d.n_replicas : 0;
    // bond planes also for the small lattices (L <= 32), which the shared-memory kernel can take
    s.bplanes = (plane_eligible(d) || d.L <= 32) ? sizeof(uint32_t) * 12 * WP : 0;
    return s;
}

// Words per thread of a streaming job: the largest of 4, 2, 1 that is at most
// max_words and divides the row's W words (chunks tile the rows exactly).
int pool_words(const Geometry &g, int max_words) {
    for (int nw = 4; nw > 1; nw >>= 1)
        if (nw <= max_words && g.W % nw == 0) return nw;
    return 1;
}

void drop_pool_graphs(micsa_pool_t p);

// Rebuild the virtual-block table and upload both tables (descriptor rows and
// vblocks) after the previous upload has been consumed.
int upload_tables(micsa_pool_t p) {
    if (!p->tables_dirty) return MICSA_OK;
    PCK(p, cudaEventSynchronize(p->tables_free), "wait for table upload");
    int nvb = 0, nunits = 0;
    // big jobs first, so that the grid-stride loop and the work counter start on the long items
    std::vector<int> order;
    for (int i = 0; i < p->max_jobs; ++i)
        if (p->slots[i].live) order.push_back(i);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        return p->slots[a].desc.L * p->slots[a].desc.n_replicas > p->slots[b].desc.L * p->slots[b].desc.n_replicas;
    });
    int npvb = 0, npu = 0;
    std::vector<PlaneUnit> units_c[kMaxCluster + 1];  // the shared-memory units by cluster size
    size_t unit_smem[kMaxCluster + 1] = {};
    for (int i : order) {
        const JobDesc &J = p->h_jobs[i];
        if (J.resident) {
            for (int r = 0; r < J.R; ++r) {
                if (nunits >= p->max_units) return pfail(p, MICSA_E_BUSY, "resident unit table full");
                p->h_units[nunits++] = ResidentUnit{J.spins + (int64_t)r * 2 * J.geo.half,
                                                    J.daemons + (int64_t)r * 2 * J.geo.half, J.bonds, r, i};
            }
        }
    }
    // byte-layout virtual blocks: the byte-streamed jobs first (their half-sweeps
    // run over this part), then the bit-plane jobs (measured over it after the tick)
    for (int pass = 0; pass < 2; ++pass)
        for (int i : order) {
            const JobDesc &J = p->h_jobs[i];
            if (J.resident || (J.use_planes != 0) != (pass == 1)) continue;
            const int64_t chunks = (int64_t)J.geo.L * J.geo.L * (J.geo.W / J.nw);
            for (int r = 0; r < J.R; ++r)
                for (int64_t c = 0; c < chunks; c += kVBlock) {
                    if (nvb >= p->max_vblocks) return pfail(p, MICSA_E_BUSY, "virtual block table full");
                    p->h_vblocks[nvb++] = VBlock{i, (int16_t)r, 0, (int32_t)c};
                }
            if (pass == 1 && J.smem_planes) {
                // one CTA per unit (C = 1; small lattices: C = 0, CTAs of 128 threads), or a
                // cluster of C CTAs holding one z word each
                const int C = J.geo.L <= 32 ? 0 : J.smem_cluster > 1 ? J.smem_cluster : 1;
                const int64_t words = C > 1 ? (int64_t)J.geo.L * J.geo.P : msg_plane_words(J.geo);
                const SplaneSplit sp = splane_split(words, J.R, J.smem_planes);
                for (int r0 = 0; r0 < J.R; r0 += sp.nrep) {
                    if (npu >= p->max_punits) return pfail(p, MICSA_E_BUSY, "plane unit table full");
                    units_c[C].push_back(PlaneUnit{i, (int16_t)r0, (int16_t)std::min(sp.nrep, J.R - r0),
                                                   (int16_t)(sp.bonds_smem ? 1 : 0), (int16_t)C});
                    unit_smem[C] = std::max(unit_smem[C], sp.bytes);
                    ++npu;
                }
            } else if (pass == 1) {
                const int64_t threads = msg_plane_words(J.geo) / 4;  // 4 plane words each
                for (int64_t c = 0; c < threads; c += kVBlock) {
                    if (npvb >= p->max_pvblocks) return pfail(p, MICSA_E_BUSY, "plane block table full");
                    p->h_pvblocks[npvb++] = PVBlock{i, (int32_t)c};
                }
            }
        }
    // the shared-memory units longest first (site updates per sweep, L^3 x replicas), so
    // that the persistent kernels' work counter hands them out in that order and the
    // tick ends close to its longest unit
    for (int C = 0; C <= kMaxCluster; ++C)
        std::stable_sort(units_c[C].begin(), units_c[C].end(), [&](const PlaneUnit &a, const PlaneUnit &b) {
            const int64_t La = p->h_jobs[a.slot].geo.L, Lb = p->h_jobs[b.slot].geo.L;
            return La * La * La * a.nrep > Lb * Lb * Lb * b.nrep;
        });
    int nvb_stream = 0;
    for (int i = 0; i < nvb; ++i)
        if (!p->h_jobs[p->h_vblocks[i].slot].use_planes) nvb_stream = i + 1;
    // the chains' parts of the byte-streamed jobs: ends at the (job, replica)
    // boundaries nearest c * nvb_stream / chains
    std::vector<int> bounds;
    for (int v = 0; v <= nvb_stream; ++v)
        if (v == 0 || v == nvb_stream || p->h_vblocks[v].slot != p->h_vblocks[v - 1].slot ||
            p->h_vblocks[v].replica != p->h_vblocks[v - 1].replica)
            bounds.push_back(v);
    int prev = 0;
    for (int c = 0; c < kPoolMaxChains; ++c) {
        int end = nvb_stream;
        if (c + 1 < p->chains) {
            const double target = (double)(c + 1) * nvb_stream / p->chains;
            int best = nvb_stream;
            for (int v : bounds)
                if (v >= prev && std::fabs(v - target) < std::fabs(best - target)) best = v;
            end = best;
        }
        p->h_nvb[c] = end;
        prev = end;
    }
    p->h_nvb[kPoolMaxChains] = nvb;
    // the bit-plane jobs' parts, split the same way at job boundaries
    std::vector<int> pbounds;
    for (int v = 0; v <= npvb; ++v)
        if (v == 0 || v == npvb || p->h_pvblocks[v].slot != p->h_pvblocks[v - 1].slot) pbounds.push_back(v);
    prev = 0;
    for (int c = 0; c < kPoolMaxChains; ++c) {
        int end = npvb;
        if (c + 1 < p->chains) {
            const double target = (double)(c + 1) * npvb / p->chains;
            int best = npvb;
            for (int v : pbounds)
                if (v >= prev && std::fabs(v - target) < std::fabs(best - target)) best = v;
            end = best;
        }
        p->h_npvb[c] = end;
        prev = end;
    }
    *p->h_nunits = nunits;
    // the table by cluster size (each kernel reads its own range); a change of
    // any launch's shared memory invalidates the captured ticks
    int at = 0;
    bool smem_changed = false;
    for (int C = 0; C <= kMaxCluster; ++C) {
        p->h_pustart[C] = at;
        p->h_npunits[C] = (int32_t)units_c[C].size();
        for (const PlaneUnit &U : units_c[C]) p->h_punits[at++] = U;
        if (unit_smem[C] != p->splanes_launch_smem[C]) {
            p->splanes_launch_smem[C] = unit_smem[C];
            smem_changed = true;
        }
    }
    if (smem_changed) drop_pool_graphs(p);
    p->has_stream_jobs = nvb_stream > 0;
    p->has_resident_jobs = nunits > 0;
    p->has_plane_jobs = npvb > 0;
    std::memcpy(p->h_jobs_stage, p->h_jobs.data(), sizeof(JobDesc) * p->max_jobs);
    PCK(p, cudaMemcpyAsync(p->d_jobs, p->h_jobs_stage, sizeof(JobDesc) * p->max_jobs, cudaMemcpyHostToDevice, p->stream), "upload jobs");
    PCK(p, cudaMemcpyAsync(p->d_vblocks, p->h_vblocks, sizeof(VBlock) * (size_t)(nvb ? nvb : 1), cudaMemcpyHostToDevice, p->stream), "upload vblocks");
    PCK(p, cudaMemcpyAsync(p->d_nvb, p->h_nvb, (kPoolMaxChains + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, p->stream), "upload vblock counts");
    PCK(p, cudaMemcpyAsync(p->d_pvblocks, p->h_pvblocks, sizeof(PVBlock) * (size_t)(npvb ? npvb : 1), cudaMemcpyHostToDevice, p->stream), "upload plane blocks");
    PCK(p, cudaMemcpyAsync(p->d_npvb, p->h_npvb, kPoolMaxChains * sizeof(int32_t), cudaMemcpyHostToDevice, p->stream), "upload plane block counts");
    if (p->max_units) {
        PCK(p, cudaMemcpyAsync(p->d_units, p->h_units, sizeof(ResidentUnit) * (size_t)(nunits ? nunits : 1), cudaMemcpyHostToDevice, p->stream), "upload units");
        PCK(p, cudaMemcpyAsync(p->d_nunits, p->h_nunits, sizeof(int32_t), cudaMemcpyHostToDevice, p->stream), "upload unit count");
    }
    PCK(p, cudaMemcpyAsync(p->d_punits, p->h_punits, sizeof(PlaneUnit) * (size_t)(npu ? npu : 1), cudaMemcpyHostToDevice, p->stream), "upload plane units");
    PCK(p, cudaMemcpyAsync(p->d_npunits, p->h_npunits, sizeof(int32_t) * (kMaxCluster + 1), cudaMemcpyHostToDevice, p->stream), "upload plane unit counts");
    PCK(p, cudaMemcpyAsync(p->d_pustart, p->h_pustart, sizeof(int32_t) * (kMaxCluster + 1), cudaMemcpyHostToDevice, p->stream), "upload plane unit starts");
    PCK(p, cudaEventRecord(p->tables_free, p->stream), "record table event");
    p->tables_dirty = false;
    return MICSA_OK;
}

// One tick: the resident kernel (mask bit 0) runs K sweeps of every job that
// lives in shared memory and measures it; the streaming half-sweeps (bit 1)
// run K sweeps of the other jobs, which the measure kernel then measures; the
// advance kernel moves every job's clock.
int enqueue_tick(micsa_pool_t p, cudaStream_t st, int mask) {
    long long *R0 = p->d_results;
    const size_t rows = (size_t)p->max_jobs * kPoolMaxR;
    PoolTables T{p->d_jobs, p->d_vblocks, p->d_nvb, p->d_pvblocks, p->d_npvb, R0, R0 + rows, R0 + 2 * rows,
                 R0 + 3 * rows, p->d_acc, p->d_improved};
    const bool resident = (mask & 1) && p->resident_smem, streamed = (mask & 2) != 0, planes = (mask & 4) != 0;
    // the resident kernel runs on a forked branch, concurrently with the other
    // parts (they touch disjoint jobs), joined before the advance node
    const bool fork = resident && (streamed || planes);
    cudaStream_t rs = st;
    if (fork) {
        PCK(p, cudaEventRecord(p->fork_ev, st), "fork event");
        PCK(p, cudaStreamWaitEvent(p->aux_stream, p->fork_ev, 0), "fork wait");
        rs = p->aux_stream;
    }
    // the bit-plane jobs held in shared memory: one persistent launch per cluster
    // size present (bit 8 << (C - 1) of the mask), each on its own branch
    const bool splanes = (mask & (((1 << (kMaxCluster + 1)) - 1) << 3)) != 0;
    if (splanes) PCK(p, cudaEventRecord(p->splanes_fork, st), "smem planes fork event");
    for (int C = 1; C <= kMaxCluster + 1; ++C) {
        if (!(mask & (8 << (C - 1)))) continue;
        cudaStream_t ss = p->splanes_stream[C];
        PCK(p, cudaStreamWaitEvent(ss, p->splanes_fork, 0), "smem planes fork wait");
        int K = p->K;
        void *args[] = {&T, &p->d_punits, &p->d_pustart, &p->d_npunits, &p->d_counter, &K};
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        cfg.dynamicSmemBytes = p->splanes_launch_smem[C == kMaxCluster + 1 ? 0 : C];
        cfg.stream = ss;
        const void *fn;
        if (C == kMaxCluster + 1) {  // the small lattices
            cfg.gridDim = dim3(p->small_grid);
            cfg.blockDim = dim3(kSmallPlaneThreads);
            fn = (const void *)pool_smem_planes_kernel<kSmallPlaneThreads, kSmallPlaneBlocks, 0>;
        } else if (C == 1) {
            const bool small = p->splanes_grid > p->sm_count;  // two or more CTAs per SM
            cfg.gridDim = dim3(p->splanes_grid);
            cfg.blockDim = dim3(small ? kSmemPlaneThreadsSmall : kSmemPlaneThreads);
            fn = small ? (const void *)pool_smem_planes_kernel<kSmemPlaneThreadsSmall, 2>
                       : (const void *)pool_smem_planes_kernel<kSmemPlaneThreads, 1>;
        } else {
            cfg.gridDim = dim3(p->cluster_grid[C]);
            cfg.blockDim = dim3(kSmemPlaneThreads);
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = C;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            fn = (const void *)pool_cluster_planes_kernel<kSmemPlaneThreads>;
        }
        PCK(p, cudaLaunchKernelExC(&cfg, fn, args), "pool smem planes launch");
        PCK(p, cudaEventRecord(p->splanes_join[C], ss), "smem planes join event");
    }
    // the shared-memory multispin kernel after the longer bit-plane units: its CTAs take the
    // SMs that the bit-plane kernel leaves as its queue drains
    if (resident) {
        ResidentArgs ra{};
        ra.units = p->d_units;
        ra.n_units_dev = p->d_nunits;
        ra.K = p->K;
        ra.counter = p->d_counter;
        ra.jobs = p->d_jobs;
        ra.results = p->d_results;
        ra.max_jobs = p->max_jobs;
        PCK(p, launch_multispin(ra, true, p->resident_smem, p->resident_grid, p->pdl && !fork, rs), "pool multispin launch");
    }
    if (planes) {
        // the bit-plane jobs' parts on their own branches: bytes -> planes, the K
        // sweeps, planes -> bytes (the measurement below reads the bytes)
        PCK(p, cudaEventRecord(p->planes_fork, st), "planes fork event");
        for (int part = 0; part < p->chains; ++part) {
            cudaStream_t ps = p->planes_stream[part];
            PCK(p, cudaStreamWaitEvent(ps, p->planes_fork, 0), "planes fork wait");
            int to_planes = 1, to_bytes = 0;
            void *cin[] = {&T, &to_planes, &part};
            PCK(p, launch_pdl((const void *)pool_planes_convert_kernel, dim3(p->grid_blocks), dim3(kVBlock), ps, cin, false),
                "pool planes in");
            for (int k = 0; k < p->K; ++k)
                for (int par = 0; par < 2; ++par) {
                    void *args[] = {&T, &k, &par, &part};
                    PCK(p, launch_pdl((const void *)pool_msg_half_kernel, dim3(p->planes_grid), dim3(kVBlock), ps, args,
                                      p->pdl),
                        "pool plane half-sweep launch");
                }
            void *cout[] = {&T, &to_bytes, &part};
            PCK(p, launch_pdl((const void *)pool_planes_convert_kernel, dim3(p->grid_blocks), dim3(kVBlock), ps, cout,
                              p->pdl),
                "pool planes out");
            PCK(p, cudaEventRecord(p->planes_join[part], ps), "planes join event");
        }
    }
    if (streamed) {
        // the parts of the byte-streamed jobs as concurrent chains, joined before
        // the measurement
        PCK(p, cudaEventRecord(p->chain_fork, st), "chain fork event");
        for (int c = 1; c < p->chains; ++c)
            PCK(p, cudaStreamWaitEvent(p->chain_stream[c], p->chain_fork, 0), "chain fork wait");
        for (int part = 0; part < p->chains; ++part) {
            cudaStream_t cs = part == 0 ? st : p->chain_stream[part];
            for (int k = 0; k < p->K; ++k)
                for (int par = 0; par < 2; ++par) {
                    void *args[] = {&T, &k, &par, &part};
                    PCK(p, launch_pdl((const void *)pool_half_sweep_kernel, dim3(p->grid_blocks), dim3(kVBlock), cs, args,
                                      p->pdl && (part == 0 || k + par > 0)),
                        "pool half-sweep launch");
                }
        }
        for (int c = 1; c < p->chains; ++c) {
            PCK(p, cudaEventRecord(p->chain_join[c], p->chain_stream[c]), "chain join event");
            PCK(p, cudaStreamWaitEvent(st, p->chain_join[c], 0), "chain join wait");
        }
    }
    if (planes)
        for (int part = 0; part < p->chains; ++part)
            PCK(p, cudaStreamWaitEvent(st, p->planes_join[part], 0), "planes join wait");
    for (int C = 1; C <= kMaxCluster + 1; ++C)
        if (mask & (8 << (C - 1))) PCK(p, cudaStreamWaitEvent(st, p->splanes_join[C], 0), "smem planes join wait");
    if (streamed || planes || splanes) {
        int K = p->K;
        void *eargs[] = {&T};
        void *bargs[] = {&T, &K};
        PCK(p, launch_pdl((const void *)pool_energy_kernel, dim3(p->grid_blocks), dim3(kVBlock), st, eargs, p->pdl), "pool energy launch");
        PCK(p, launch_pdl((const void *)pool_best_kernel, dim3(p->max_jobs), dim3(32), st, bargs, p->pdl), "pool best launch");
        PCK(p, launch_pdl((const void *)pool_best_copy_kernel, dim3(p->grid_blocks), dim3(kVBlock), st, eargs, p->pdl), "pool best copy launch");
    }
    if (fork) {
        PCK(p, cudaEventRecord(p->join_ev, p->aux_stream), "join event");
        PCK(p, cudaStreamWaitEvent(st, p->join_ev, 0), "join wait");
    }
    int K = p->K, mj = p->max_jobs;
    void *aargs[] = {&p->d_jobs, &mj, &K, &p->d_counter};
    PCK(p, launch_pdl((const void *)pool_advance_kernel, dim3((p->max_jobs + 255) / 256), dim3(256), st, aargs, p->pdl && !fork), "pool advance launch");
    return MICSA_OK;
}

int tick_launches(micsa_pool_t p, int mask) {
    const int resident = (mask & 1) && p->resident_smem ? 1 : 0;
    const int streamed = (mask & 2) ? 2 * p->chains * p->K : 0;
    const int planes = (mask & 4) ? p->chains * (2 * p->K + 2) : 0;
    int splanes = 0;
    for (int C = 1; C <= kMaxCluster + 1; ++C) splanes += (mask & (8 << (C - 1))) ? 1 : 0;
    return resident + streamed + planes + splanes + ((mask & ~1) ? 3 : 0) + 1;
}

int ensure_graph(micsa_pool_t p, int mask) {
    if (p->graphs[mask] || !p->use_graph) return MICSA_OK;
    PCK(p, cudaStreamBeginCapture(p->capture_stream, cudaStreamCaptureModeThreadLocal), "pool begin capture");
    const int rc = enqueue_tick(p, p->capture_stream, mask);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(p->capture_stream, &g);
    if (rc != MICSA_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    PCK(p, e, "pool end capture");
    const cudaError_t e2 = cudaGraphInstantiate(&p->graphs[mask], g, 0);
    cudaGraphDestroy(g);
    PCK(p, e2, "pool graph instantiate");
    return MICSA_OK;
}

void drop_pool_graphs(micsa_pool_t p) {
    for (auto &g : p->graphs) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

void release_slot(micsa_pool_t p, int i) {
    PoolJob &j = p->slots[i];
    arena_free(p, j.off_bonds, j.bytes);
    j = PoolJob{};
    p->h_jobs[i] = JobDesc{};
    p->tables_dirty = true;
}

}  // namespace

extern "C" {

int micsa_pool_create(size_t arena_bytes, int max_jobs, int tick_sweeps, micsa_pool_t *out) {
    if (!out || max_jobs < 1 || max_jobs > 65535 || tick_sweeps < 1 || tick_sweeps > 4096 || arena_bytes < (1u << 20))
        return MICSA_E_INVALID_ARG;
    *out = nullptr;
    micsa_pool *p = new (std::nothrow) micsa_pool;
    if (!p) return MICSA_E_OOM;
    p->max_jobs = max_jobs;
    p->K = tick_sweeps;
    p->arena_bytes = align_up(arena_bytes);
    p->slots.resize(max_jobs);
    p->h_jobs.assign(max_jobs, JobDesc{});
    p->stage.assign(max_jobs, nullptr);
    p->stage_cap.assign(max_jobs, 0);
    p->stage_free.assign(max_jobs, nullptr);
    int rc = MICSA_OK;
    auto bail = [&](int code) { rc = code; };
    cudaError_t e = cudaSuccess;
    do {
        if ((e = cudaGetDevice(&p->device)) != cudaSuccess) { bail(MICSA_E_CUDA); break; }
        if ((e = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device)) != cudaSuccess) { bail(MICSA_E_CUDA); break; }
        if ((e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking)) != cudaSuccess) { bail(MICSA_E_CUDA); break; }
        if ((e = cudaStreamCreateWithFlags(&p->capture_stream, cudaStreamNonBlocking)) != cudaSuccess) { bail(MICSA_E_CUDA); break; }
        if ((e = cudaStreamCreateWithFlags(&p->aux_stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&p->chain_fork, cudaEventDisableTiming)) != cudaSuccess) { bail(MICSA_E_CUDA); break; }
        for (int c = 1; c < kPoolMaxChains && e == cudaSuccess; ++c)
            if ((e = cudaStreamCreateWithFlags(&p->chain_stream[c], cudaStreamNonBlocking)) == cudaSuccess)
                e = cudaEventCreateWithFlags(&p->chain_join[c], cudaEventDisableTiming);
        if (e != cudaSuccess) { bail(MICSA_E_CUDA); break; }
        if ((e = cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&p->join_ev, cudaEventDisableTiming)) != cudaSuccess) { bail(MICSA_E_CUDA); break; }
        if ((e = cudaEventCreateWithFlags(&p->tables_free, cudaEventDisableTiming)) != cudaSuccess) { bail(MICSA_E_CUDA); break; }
        if ((e = cudaMalloc(&p->arena, p->arena_bytes)) != cudaSuccess) { bail(MICSA_E_OOM); break; }
        p->free_list[0] = p->arena_bytes;
        p->max_vblocks = 1 << 22;
        p->max_pvblocks = 1 << 20;
        if ((e = cudaMalloc(&p->d_jobs, sizeof(JobDesc) * max_jobs)) != cudaSuccess ||
            (e = cudaMalloc(&p->d_vblocks, sizeof(VBlock) * (size_t)p->max_vblocks)) != cudaSuccess ||
            (e = cudaMalloc(&p->d_nvb, (kPoolMaxChains + 1) * sizeof(int32_t))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_pvblocks, sizeof(PVBlock) * (size_t)p->max_pvblocks)) != cudaSuccess ||
            (e = cudaMalloc(&p->d_npvb, kPoolMaxChains * sizeof(int32_t))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_results, sizeof(long long) * 4 * (size_t)max_jobs * kPoolMaxR)) != cudaSuccess ||
            (e = cudaMalloc(&p->d_acc, sizeof(unsigned long long) * 2 * (size_t)max_jobs * kPoolMaxR)) != cudaSuccess ||
            (e = cudaMalloc(&p->d_improved, sizeof(int32_t) * (size_t)max_jobs * kPoolMaxR)) != cudaSuccess) { bail(MICSA_E_OOM); break; }
        if ((e = cudaMemsetAsync(p->d_acc, 0, sizeof(unsigned long long) * 2 * (size_t)max_jobs * kPoolMaxR, p->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(p->d_improved, 0, sizeof(int32_t) * (size_t)max_jobs * kPoolMaxR, p->stream)) != cudaSuccess) { bail(MICSA_E_CUDA); break; }
        if ((e = cudaMallocHost(&p->h_jobs_stage, sizeof(JobDesc) * max_jobs)) != cudaSuccess ||
            (e = cudaMallocHost(&p->h_vblocks, sizeof(VBlock) * (size_t)p->max_vblocks)) != cudaSuccess ||
            (e = cudaMallocHost(&p->h_nvb, (kPoolMaxChains + 1) * sizeof(int32_t))) != cudaSuccess ||
            (e = cudaMallocHost(&p->h_pvblocks, sizeof(PVBlock) * (size_t)p->max_pvblocks)) != cudaSuccess ||
            (e = cudaMallocHost(&p->h_npvb, kPoolMaxChains * sizeof(int32_t))) != cudaSuccess) { bail(MICSA_E_OOM); break; }
        for (int c = 0; c <= kPoolMaxChains; ++c) p->h_nvb[c] = 0;
        for (int c = 0; c < kPoolMaxChains; ++c) p->h_npvb[c] = 0;
        for (auto &ev : p->stage_free)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) { bail(MICSA_E_CUDA); break; }
        if (rc) break;
        if ((e = cudaMemsetAsync(p->d_jobs, 0, sizeof(JobDesc) * max_jobs, p->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(p->d_nvb, 0, (kPoolMaxChains + 1) * sizeof(int32_t), p->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(p->d_npvb, 0, kPoolMaxChains * sizeof(int32_t), p->stream)) != cudaSuccess) { bail(MICSA_E_CUDA); break; }
        // jobs of L <= 32 live in shared memory as bit planes (multispin kernel)
        p->resident_smem = multispin_smem_bytes(make_geometry(32));
        const int res_per_sm = multispin_blocks_per_sm(true, p->resident_smem);
        if (res_per_sm <= 0) p->resident_smem = 0;
        p->resident_grid = (res_per_sm > 0 ? res_per_sm : 1) * p->sm_count;
        p->max_units = max_jobs * kPoolMaxR;
        if ((e = cudaMalloc(&p->d_units, sizeof(ResidentUnit) * (size_t)p->max_units)) != cudaSuccess ||
            (e = cudaMalloc(&p->d_nunits, sizeof(int32_t))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_counter, (kMaxCluster + 2) * sizeof(int))) != cudaSuccess ||
            (e = cudaMallocHost(&p->h_units, sizeof(ResidentUnit) * (size_t)p->max_units)) != cudaSuccess ||
            (e = cudaMallocHost(&p->h_nunits, sizeof(int32_t))) != cudaSuccess) { bail(MICSA_E_OOM); break; }
        *p->h_nunits = 0;
        if ((e = cudaMemsetAsync(p->d_nunits, 0, sizeof(int32_t), p->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(p->d_counter, 0, (kMaxCluster + 2) * sizeof(int), p->stream)) != cudaSuccess) { bail(MICSA_E_CUDA); break; }
        // bit-plane jobs in shared memory: one CTA of kSmemPlaneThreads per unit, the budget
        // the device allows a block (opt-in) less the kernel's static shared memory
        p->max_punits = max_jobs * kPoolMaxR;
        if ((e = cudaMalloc(&p->d_punits, sizeof(PlaneUnit) * (size_t)p->max_punits)) != cudaSuccess ||
            (e = cudaMalloc(&p->d_npunits, sizeof(int32_t) * (kMaxCluster + 1))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_pustart, sizeof(int32_t) * (kMaxCluster + 1))) != cudaSuccess ||
            (e = cudaMallocHost(&p->h_punits, sizeof(PlaneUnit) * (size_t)p->max_punits)) != cudaSuccess ||
            (e = cudaMallocHost(&p->h_npunits, sizeof(int32_t) * (kMaxCluster + 1))) != cudaSuccess ||
            (e = cudaMallocHost(&p->h_pustart, sizeof(int32_t) * (kMaxCluster + 1))) != cudaSuccess) { bail(MICSA_E_OOM); break; }
        for (int C = 0; C <= kMaxCluster; ++C) p->h_npunits[C] = p->h_pustart[C] = 0;
        if ((e = cudaMemsetAsync(p->d_npunits, 0, sizeof(int32_t) * (kMaxCluster + 1), p->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(p->d_pustart, 0, sizeof(int32_t) * (kMaxCluster + 1), p->stream)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&p->splanes_fork, cudaEventDisableTiming)) != cudaSuccess) { bail(MICSA_E_CUDA); break; }
        for (int C = 1; C <= kMaxCluster + 1 && e == cudaSuccess; ++C)
            if ((e = cudaStreamCreateWithFlags(&p->splanes_stream[C], cudaStreamNonBlocking)) == cudaSuccess)
                e = cudaEventCreateWithFlags(&p->splanes_join[C], cudaEventDisableTiming);
        if (e != cudaSuccess) { bail(MICSA_E_CUDA); break; }
        {
            int optin = 0;
            cudaFuncAttributes fa{};
            if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device)) != cudaSuccess ||
                (e = cudaFuncGetAttributes(&fa, pool_smem_planes_kernel<kSmemPlaneThreads, 1>)) != cudaSuccess) { bail(MICSA_E_CUDA); break; }
            p->splanes_max_smem = (size_t)optin > fa.sharedSizeBytes ? ((size_t)optin - fa.sharedSizeBytes) / 16 * 16 : 0;
            if (p->splanes_max_smem &&
                ((e = cudaFuncSetAttribute(pool_smem_planes_kernel<kSmemPlaneThreads, 1>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->splanes_max_smem)) != cudaSuccess ||
                 (e = cudaFuncSetAttribute(pool_smem_planes_kernel<kSmemPlaneThreadsSmall, 2>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->splanes_max_smem)) != cudaSuccess)) {
                bail(MICSA_E_CUDA);
                break;
            }
            p->splanes_smem = p->splanes_max_smem;
            p->splanes_grid = p->sm_count;  // one CTA per SM at the full budget
            if (p->splanes_max_smem &&
                ((e = cudaFuncSetAttribute(pool_cluster_planes_kernel<kSmemPlaneThreads>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->splanes_max_smem)) != cudaSuccess ||
                 (e = cudaFuncSetAttribute(pool_smem_planes_kernel<kSmallPlaneThreads, kSmallPlaneBlocks, 0>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallPlaneSmem)) != cudaSuccess)) {
                bail(MICSA_E_CUDA);
                break;
            }
            p->small_grid = kSmallPlaneBlocks * p->sm_count;
            // clusters of C CTAs (one per SM at the full budget) that can be resident at once
            for (int C = 2; C <= kMaxCluster; ++C) {
                cudaLaunchConfig_t cfg = {};
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = C;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.gridDim = dim3((unsigned)(p->sm_count / C * C));
                cfg.blockDim = dim3(kSmemPlaneThreads);
                cfg.dynamicSmemBytes = p->splanes_max_smem;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                int clusters = 0;
                if (cudaOccupancyMaxActiveClusters(&clusters, (const void *)pool_cluster_planes_kernel<kSmemPlaneThreads>,
                                                   &cfg) != cudaSuccess || clusters < 1) {
                    cudaGetLastError();  // not fatal: fall back to one cluster per C SMs
                    clusters = p->sm_count / C;
                }
                p->cluster_grid[C] = std::max(1, clusters) * C;
            }
        }
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pool_half_sweep_kernel, kVBlock, 0);
        int per_sm_planes = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_planes, pool_msg_half_kernel, kVBlock, 0);
        p->planes_grid = (per_sm_planes > 0 ? per_sm_planes : 4) * p->sm_count;
        if ((e = cudaEventCreateWithFlags(&p->planes_fork, cudaEventDisableTiming)) != cudaSuccess) { bail(MICSA_E_CUDA); break; }
        for (int c = 0; c < kPoolMaxChains && e == cudaSuccess; ++c)
            if ((e = cudaStreamCreateWithFlags(&p->planes_stream[c], cudaStreamNonBlocking)) == cudaSuccess)
                e = cudaEventCreateWithFlags(&p->planes_join[c], cudaEventDisableTiming);
        if (e != cudaSuccess) { bail(MICSA_E_CUDA); break; }
        p->grid_blocks = (per_sm > 0 ? per_sm : 4) * p->sm_count;
        p->tick_events.resize(64);
        for (auto &ev : p->tick_events)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) { bail(MICSA_E_CUDA); break; }
        if (rc) break;
        if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess) { bail(MICSA_E_CUDA); break; }
    } while (0);
    if (rc != MICSA_OK) p->err = std::string("pool creation failed: ") + cudaGetErrorString(e);
    if (rc != MICSA_OK) {
        micsa_pool_destroy(p);
        return rc;
    }
    *out = p;
    return MICSA_OK;
}

void micsa_pool_destroy(micsa_pool_t p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    drop_pool_graphs(p);
    for (auto ev : p->tick_events)
        if (ev) cudaEventDestroy(ev);
    for (auto *b : p->stage) cudaFreeHost(b);
    for (auto ev : p->stage_free)
        if (ev) cudaEventDestroy(ev);
    if (p->tables_free) cudaEventDestroy(p->tables_free);
    cudaFree(p->arena);
    cudaFree(p->d_jobs);
    cudaFree(p->d_vblocks);
    cudaFree(p->d_nvb);
    cudaFree(p->d_results);
    cudaFree(p->d_acc);
    cudaFree(p->d_improved);
    cudaFreeHost(p->h_jobs_stage);
    cudaFree(p->d_units);
    cudaFree(p->d_nunits);
    cudaFree(p->d_counter);
    cudaFree(p->d_punits);
    cudaFree(p->d_npunits);
    cudaFree(p->d_pustart);
    cudaFreeHost(p->h_punits);
    cudaFreeHost(p->h_npunits);
    cudaFreeHost(p->h_pustart);
    for (int C = 1; C <= kMaxCluster + 1; ++C) {
        if (p->splanes_stream[C]) {
            cudaStreamSynchronize(p->splanes_stream[C]);
            cudaStreamDestroy(p->splanes_stream[C]);
        }
        if (p->splanes_join[C]) cudaEventDestroy(p->splanes_join[C]);
    }
    if (p->splanes_fork) cudaEventDestroy(p->splanes_fork);
    cudaFreeHost(p->h_units);
    cudaFreeHost(p->h_nunits);
    cudaFreeHost(p->h_vblocks);
    cudaFreeHost(p->h_nvb);
    cudaFree(p->d_pvblocks);
    cudaFree(p->d_npvb);
    cudaFreeHost(p->h_pvblocks);
    cudaFreeHost(p->h_npvb);
    for (int c = 0; c < kPoolMaxChains; ++c) {
        if (p->planes_stream[c]) {
            cudaStreamSynchronize(p->planes_stream[c]);
            cudaStreamDestroy(p->planes_stream[c]);
        }
        if (p->planes_join[c]) cudaEventDestroy(p->planes_join[c]);
    }
    if (p->planes_fork) cudaEventDestroy(p->planes_fork);
    if (p->capture_stream) cudaStreamDestroy(p->capture_stream);
    if (p->aux_stream) {
        cudaStreamSynchronize(p->aux_stream);
        cudaStreamDestroy(p->aux_stream);
    }
    if (p->fork_ev) cudaEventDestroy(p->fork_ev);
    if (p->join_ev) cudaEventDestroy(p->join_ev);
    for (int c = 0; c < kPoolMaxChains; ++c) {
        if (p->chain_stream[c]) {
            cudaStreamSynchronize(p->chain_stream[c]);
            cudaStreamDestroy(p->chain_stream[c]);
        }
        if (p->chain_join[c]) cudaEventDestroy(p->chain_join[c]);
    }
    if (p->chain_fork) cudaEventDestroy(p->chain_fork);
    if (p->stream) cudaStreamDestroy(p->stream);
    delete p;
}

const char *micsa_pool_last_error(micsa_pool_t p) { return p ? p->err.c_str() : "invalid pool (NULL)"; }

int micsa_pool_job_bytes(const micsa_job_desc *job, size_t *bytes) {
    if (!job || !bytes) return MICSA_E_INVALID_ARG;
    const JobSizes s = job_sizes(*job);
    *bytes = align_up(s.bonds) + 2 * align_up(s.state) + align_up(s.best) + align_up(s.thr) + align_up(s.planes) +
             align_up(s.bplanes);
    return MICSA_OK;
}

int micsa_pool_submit(micsa_pool_t p, const micsa_job_desc *job, int64_t *job_id) {
    if (!p || !job || !job_id) return MICSA_E_INVALID_ARG;
    const micsa_job_desc d = *job;
    if (d.L < 2 || d.L > 1024 || (d.L & 1) || d.n_replicas < 1 || d.n_replicas > kPoolMaxR || d.n_sweeps < 1 ||
        d.refresh_interval < 1 || !(d.T_start > 0.0) || !(d.T_end > 0.0) || !std::isfinite(d.T_start) ||
        !std::isfinite(d.T_end))
        return pfail(p, MICSA_E_INVALID_ARG, "bad job description");
    int slot = -1;
    for (int i = 0; i < p->max_jobs; ++i)
        if (p->slots[i].id < 0) { slot = i; break; }
    if (slot < 0) return pfail(p, MICSA_E_BUSY, "no free slot");
    const JobSizes s = job_sizes(d);
    size_t total = 0;
    micsa_pool_job_bytes(&d, &total);
    size_t off = 0;
    if (!arena_alloc(p, total, &off)) return pfail(p, MICSA_E_BUSY, "arena has no %zu free bytes", total);
    PoolJob &J = p->slots[slot];
    J.id = p->next_id++;
    J.desc = d;
    J.bytes = total;
    J.off_bonds = off;
    J.off_spins = J.off_bonds + align_up(s.bonds);
    J.off_daemons = J.off_spins + align_up(s.state);
    J.off_best = J.off_daemons + align_up(s.state);
    J.off_thr = J.off_best + align_up(s.best);
    J.off_planes = J.off_thr + align_up(s.thr);
    J.off_bplanes = J.off_planes + align_up(s.planes);
    J.t = 0;
    J.live = true;
    J.done_tick = -1;
    // refresh cut points for every refresh of the job (ordinal j at sweep
    // j * interval) and the reset values of its result rows, staged in pinned
    // memory so that nothing here waits for the queued ticks
    const size_t need = s.thr + sizeof(long long) * 4 * kPoolMaxR;
    if (p->stage_cap[slot] < need) {
        PCK(p, cudaEventSynchronize(p->stage_free[slot]), "staging reuse");
        cudaFreeHost(p->stage[slot]);
        p->stage[slot] = nullptr;
        p->stage_cap[slot] = 0;
        PCK(p, cudaMallocHost(&p->stage[slot], need), "pinned job staging");
        p->stage_cap[slot] = need;
    } else {
        PCK(p, cudaEventSynchronize(p->stage_free[slot]), "staging reuse");
    }
    uint64_t *thr = p->stage[slot];
    for (int64_t j = 0; j < s.n_refresh; ++j)
        micsa_daemon_thresholds(schedule_T(d, j * (int64_t)d.refresh_interval), thr + 3 * j);
    long long *init = reinterpret_cast<long long *>(reinterpret_cast<uint8_t *>(thr) + s.thr);
    for (int q = 0; q < 4; ++q)
        for (int r = 0; r < kPoolMaxR; ++r) init[q * kPoolMaxR + r] = (q == 2) ? (1ll << 62) : 0;
    uint8_t *base = p->arena;
    PCK(p, cudaMemcpyAsync(base + J.off_thr, thr, s.thr, cudaMemcpyHostToDevice, p->stream), "upload thresholds");
    for (int q = 0; q < 4; ++q)
        PCK(p, cudaMemcpyAsync(p->d_results + (size_t)q * p->max_jobs * kPoolMaxR + (size_t)slot * kPoolMaxR,
                               init + q * kPoolMaxR, sizeof(long long) * kPoolMaxR, cudaMemcpyHostToDevice, p->stream),
            "reset results");
    PCK(p, cudaEventRecord(p->stage_free[slot], p->stream), "record staging event");
    PCK(p, cudaMemsetAsync(base + J.off_bonds, 0, s.bonds, p->stream), "clear bonds");
    PCK(p, cudaMemsetAsync(base + J.off_spins, 0, s.state, p->stream), "clear spins");
    PCK(p, cudaMemsetAsync(base + J.off_daemons, 0, s.state, p->stream), "clear daemons");
    const uint32_t k0 = (uint32_t)(d.seed & 0xFFFFFFFFu), k1 = (uint32_t)(d.seed >> 32);
    PCK(p, launch_init_couplings(base + J.off_bonds, s.g, 1, k0, k1, p->stream), "job couplings");
    PCK(p, launch_init_spins(reinterpret_cast<int8_t *>(base + J.off_spins), s.g, 1, d.n_replicas, k0, k1, p->stream), "job spins");
    p->launches += 2;
    JobDesc &D = p->h_jobs[slot];
    D.spins = reinterpret_cast<int8_t *>(base + J.off_spins);
    D.daemons = base + J.off_daemons;
    D.bonds = base + J.off_bonds;
    D.best = reinterpret_cast<int8_t *>(base + J.off_best);
    D.thr = reinterpret_cast<const uint64_t *>(base + J.off_thr);
    D.geo = s.g;
    D.R = d.n_replicas;
    D.nw = pool_words(s.g, p->max_words);
    D.key0 = k0;
    D.key1 = k1;
    D.t = 0;
    D.n_sweeps = d.n_sweeps;
    D.interval = d.refresh_interval;
    D.live = 1;
    const FastDiv fdL = make_fastdiv((uint32_t)d.L);
    D.divL_m = fdL.m;
    D.divL_l = fdL.l;
    const FastDiv fdC = make_fastdiv((uint32_t)(s.g.W / D.nw));
    D.divC_m = fdC.m;
    D.divC_l = fdC.l;
    // L <= 32: bit planes in shared memory (units of a few replicas in CTAs of 128
    // threads) when on, else the multispin kernel
    const bool small_planes = p->small_planes && p->splanes_max_smem && d.L <= 32;
    D.resident = (!small_planes && p->resident_smem && multispin_smem_bytes(s.g) &&
                  multispin_smem_bytes(s.g) <= p->resident_smem) ? 1 : 0;
    D.use_planes = ((p->planes_on && plane_eligible(d) && !D.resident) || small_planes) ? 1 : 0;
    // shared memory: split over a cluster of one CTA per z word when on and a
    // replica's slice fits, else the whole unit in one CTA when a replica fits
    const int nzw = (d.L + 31) / 32;
    D.smem_cluster = 0;
    D.smem_planes = 0;
    if (small_planes) {
        D.smem_planes = (int32_t)kSmallPlaneSmem;
    } else if (D.use_planes && p->splanes_cluster && nzw >= 2 && nzw <= kMaxCluster &&
        splane_split((int64_t)d.L * s.g.P, d.n_replicas, p->splanes_smem).nrep > 0) {
        D.smem_cluster = nzw;
        D.smem_planes = (int32_t)p->splanes_smem;
    } else if (D.use_planes && splane_split(msg_plane_words(s.g), d.n_replicas, p->splanes_smem).nrep > 0) {
        D.smem_planes = (int32_t)p->splanes_smem;
    }
    D.planes = D.use_planes ? reinterpret_cast<uint32_t *>(base + J.off_planes) : nullptr;
    D.bplanes = D.use_planes ? reinterpret_cast<const uint32_t *>(base + J.off_bplanes) : nullptr;
    if (D.use_planes) {  // the bonds never change: their planes are made once
        PCK(p, msg_convert_bonds(reinterpret_cast<uint32_t *>(base + J.off_bplanes), base + J.off_bonds, s.g, 1,
                                 p->stream),
            "job bond planes");
        ++p->launches;
    }
    p->tables_dirty = true;
    *job_id = J.id;
    return MICSA_OK;
}

int micsa_pool_tick(micsa_pool_t p) {
    if (!p) return MICSA_E_INVALID_ARG;
    if (int rc = upload_tables(p)) return rc;
    int mask = (p->has_resident_jobs ? 1 : 0) | (p->has_stream_jobs ? 2 : 0) | (p->has_plane_jobs ? 4 : 0);
    for (int C = 1; C <= kMaxCluster; ++C) mask |= p->h_npunits[C] > 0 ? (8 << (C - 1)) : 0;
    mask |= p->h_npunits[0] > 0 ? (8 << kMaxCluster) : 0;  // the small lattices
    if (int rc = ensure_graph(p, mask)) return rc;
    if (p->graphs[mask]) {
        PCK(p, cudaGraphLaunch(p->graphs[mask], p->stream), "pool graph launch");
    } else {
        if (int rc = enqueue_tick(p, p->stream, mask)) return rc;
    }
    p->launches += tick_launches(p, mask);
    const int64_t tick = p->ticks_queued++;
    cudaEvent_t ev = p->tick_events[tick % p->tick_events.size()];
    if (tick >= (int64_t)p->tick_events.size())
        PCK(p, cudaEventSynchronize(ev), "tick event reuse");  // bounds the ticks in flight
    PCK(p, cudaEventRecord(ev, p->stream), "record tick event");
    for (int i = 0; i < p->max_jobs; ++i) {
        PoolJob &J = p->slots[i];
        if (!J.live || J.done_tick >= 0) continue;
        J.t = std::min<int64_t>(J.t + p->K, J.desc.n_sweeps);
        p->h_jobs[i].t = J.t;  // what the tick's advance kernel will leave on the device
        if (J.t >= J.desc.n_sweeps) J.done_tick = tick;
    }
    return MICSA_OK;
}

int micsa_pool_wait(micsa_pool_t p) {
    if (!p) return MICSA_E_INVALID_ARG;
    PCK(p, cudaStreamSynchronize(p->stream), "pool synchronize");
    return MICSA_OK;
}

int micsa_pool_wait_ticks(micsa_pool_t p, int max_pending) {
    if (!p || max_pending < 0) return MICSA_E_INVALID_ARG;
    const int64_t ring = (int64_t)p->tick_events.size();
    for (int64_t tick = p->ticks_queued - 1 - max_pending; tick >= 0 && tick > p->ticks_queued - 1 - ring; --tick) {
        // ticks complete in order: waiting for the newest one that must be done suffices
        PCK(p, cudaEventSynchronize(p->tick_events[tick % ring]), "tick event");
        break;
    }
    return MICSA_OK;
}

namespace {

// Split layout [R][parity][z][y][P bytes] (byte i of row (z, y) of parity p is
// the site x = 2i + ((p + y + z) & 1)) to natural layout [R][N] on the host.
void split_to_natural(const uint8_t *split, int R, const Geometry &g, uint8_t *out) {
    const int L = g.L;
    const size_t N = (size_t)L * L * L;
    for (int r = 0; r < R; ++r)
        for (int par = 0; par < 2; ++par)
            for (int z = 0; z < L; ++z)
                for (int y = 0; y < L; ++y) {
                    const uint8_t *row = split + ((size_t)r * 2 + par) * g.half + ((size_t)z * L + y) * g.P;
                    uint8_t *o = out + (size_t)r * N + ((size_t)z * L + y) * L + ((par + y + z) & 1);
                    for (int i = 0; i < g.Lh; ++i) o[2 * i] = row[i];
                }
}

}  // namespace

int micsa_pool_poll(micsa_pool_t p, int64_t job_id, micsa_job_result *res, int8_t *best_spins) {
    return micsa_pool_poll_state(p, job_id, res, best_spins, nullptr, nullptr);
}

int micsa_pool_poll_state(micsa_pool_t p, int64_t job_id, micsa_job_result *res, int8_t *best_spins,
                          int8_t *spins, uint8_t *daemons) {
    if (!p) return MICSA_E_INVALID_ARG;
    int slot = -1;
    for (int i = 0; i < p->max_jobs; ++i)
        if (p->slots[i].id == job_id) { slot = i; break; }
    if (slot < 0) return pfail(p, MICSA_E_NOT_FOUND, "unknown job %lld", (long long)job_id);
    PoolJob &J = p->slots[slot];
    if (J.done_tick < 0) return MICSA_E_BUSY;
    cudaEvent_t ev = p->tick_events[J.done_tick % p->tick_events.size()];
    if (J.done_tick + (int64_t)p->tick_events.size() > p->ticks_queued - 1) {
        const cudaError_t q = cudaEventQuery(ev);
        if (q == cudaErrorNotReady) return MICSA_E_BUSY;
        PCK(p, q, "tick event query");
    } else {
        PCK(p, cudaEventSynchronize(ev), "tick event");  // event slot reused: wait on it via the stream order
    }
    const int R = J.desc.n_replicas;
    long long vals[4][kPoolMaxR];
    for (int q = 0; q < 4; ++q)
        PCK(p, cudaMemcpy(vals[q], p->d_results + (size_t)q * p->max_jobs * kPoolMaxR + (size_t)slot * kPoolMaxR,
                          sizeof(long long) * kPoolMaxR, cudaMemcpyDeviceToHost), "copy results");
    const Geometry g = p->h_jobs[slot].geo;
    std::vector<uint8_t> split;
    if (best_spins || spins || daemons) split.resize((size_t)R * 2 * g.half);
    if (best_spins) {
        const size_t N = (size_t)g.L * g.L * g.L;
        if (p->h_jobs[slot].resident) {  // kept in natural layout by the shared-memory kernel
            PCK(p, cudaMemcpy(best_spins, p->arena + J.off_best, (size_t)R * N, cudaMemcpyDeviceToHost), "copy best spins");
        } else {
            PCK(p, cudaMemcpy(split.data(), p->arena + J.off_best, split.size(), cudaMemcpyDeviceToHost), "copy best spins");
            split_to_natural(split.data(), R, g, reinterpret_cast<uint8_t *>(best_spins));
        }
    }
    // the final state: split layout for every job between ticks (bit-plane jobs
    // are converted back at the end of each tick)
    if (spins) {
        PCK(p, cudaMemcpy(split.data(), p->arena + J.off_spins, split.size(), cudaMemcpyDeviceToHost), "copy spins");
        split_to_natural(split.data(), R, g, reinterpret_cast<uint8_t *>(spins));
    }
    if (daemons) {
        PCK(p, cudaMemcpy(split.data(), p->arena + J.off_daemons, split.size(), cudaMemcpyDeviceToHost), "copy daemons");
        split_to_natural(split.data(), R, g, daemons);
    }
    if (res) {
        std::memset(res, 0, sizeof(*res));
        res->job_id = J.id;
        res->sweeps_done = J.desc.n_sweeps;
        res->n_replicas = R;
        for (int r = 0; r < R; ++r) {
            res->energy[r] = vals[0][r];
            res->aux[r] = vals[1][r];
            res->best_energy[r] = vals[2][r];
            res->best_t[r] = vals[3][r];
        }
    }
    // the slot's device memory may be reused only after its last tick has run
    release_slot(p, slot);
    return MICSA_OK;
}

int micsa_pool_finished(micsa_pool_t p, int64_t *ids, int max_ids, int *n_ids) {
    if (!p || !n_ids || max_ids < 0 || (max_ids > 0 && !ids)) return MICSA_E_INVALID_ARG;
    int n = 0;
    const int64_t ring = (int64_t)p->tick_events.size();
    for (int i = 0; i < p->max_jobs && n < max_ids; ++i) {
        const PoolJob &J = p->slots[i];
        if (J.id < 0 || J.done_tick < 0) continue;
        bool done = true;
        if (J.done_tick + ring > p->ticks_queued - 1) {  // its event has not been reused: ask it
            const cudaError_t q = cudaEventQuery(p->tick_events[J.done_tick % ring]);
            if (q == cudaErrorNotReady) done = false;
            else PCK(p, q, "tick event query");
        }
        if (done) ids[n++] = J.id;
    }
    *n_ids = n;
    return MICSA_OK;
}

int micsa_pool_stats(micsa_pool_t p, int *live_jobs, size_t *free_bytes, int64_t *launches) {
    if (!p) return MICSA_E_INVALID_ARG;
    if (live_jobs) {
        int n = 0;
        for (auto &j : p->slots) n += j.id >= 0;
        *live_jobs = n;
    }
    if (free_bytes) *free_bytes = arena_free_bytes(p);
    if (launches) *launches = p->launches;
    return MICSA_OK;
}

int micsa_pool_set_launch_config(micsa_pool_t p, int blocks_per_sm, int pdl, int use_graph) {
    if (!p || blocks_per_sm < 0 || blocks_per_sm > 64) return MICSA_E_INVALID_ARG;
    PCK(p, cudaStreamSynchronize(p->stream), "synchronize before reconfiguring");
    drop_pool_graphs(p);
    if (blocks_per_sm == 0) {  // as many as fit
        PCK(p, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, pool_half_sweep_kernel, kVBlock, 0),
            "occupancy query");
        if (blocks_per_sm < 1) blocks_per_sm = 4;
    }
    p->grid_blocks = blocks_per_sm * p->sm_count;
    p->pdl = pdl != 0;
    p->use_graph = use_graph != 0;
    return MICSA_OK;
}

int micsa_pool_set_planes(micsa_pool_t p, int on) {
    if (!p) return MICSA_E_INVALID_ARG;
    p->planes_on = on != 0;
    return MICSA_OK;
}

int micsa_pool_set_smem_planes(micsa_pool_t p, size_t smem_bytes, int blocks_per_sm) {
    if (!p || blocks_per_sm < 1 || blocks_per_sm > 8) return MICSA_E_INVALID_ARG;
    if (smem_bytes > p->splanes_max_smem)
        return pfail(p, MICSA_E_INVALID_ARG, "shared-memory budget %zu above the device's %zu bytes", smem_bytes,
                     p->splanes_max_smem);
    PCK(p, cudaStreamSynchronize(p->stream), "synchronize before reshaping");
    drop_pool_graphs(p);
    p->splanes_smem = smem_bytes / 16 * 16;
    p->splanes_grid = blocks_per_sm * p->sm_count;
    return MICSA_OK;
}

int micsa_pool_set_smem_clusters(micsa_pool_t p, int on) {
    if (!p) return MICSA_E_INVALID_ARG;
    p->splanes_cluster = on != 0;
    return MICSA_OK;
}

int micsa_pool_set_small_planes(micsa_pool_t p, int on) {
    if (!p) return MICSA_E_INVALID_ARG;
    p->small_planes = on != 0;
    return MICSA_OK;
}

int micsa_pool_get_smem_planes(micsa_pool_t p, size_t *smem_bytes, size_t *max_smem_bytes, int *blocks_per_sm) {
    if (!p) return MICSA_E_INVALID_ARG;
    if (smem_bytes) *smem_bytes = p->splanes_smem;
    if (max_smem_bytes) *max_smem_bytes = p->splanes_max_smem;
    if (blocks_per_sm) *blocks_per_sm = p->splanes_grid / (p->sm_count > 0 ? p->sm_count : 1);
    return MICSA_OK;
}

int micsa_pool_set_shape(micsa_pool_t p, int max_words, int chains) {
    if (!p || (max_words != 1 && max_words != 2 && max_words != 4) || chains < 1 || chains > kPoolMaxChains)
        return MICSA_E_INVALID_ARG;
    PCK(p, cudaStreamSynchronize(p->stream), "synchronize before reshaping");
    drop_pool_graphs(p);
    p->max_words = max_words;
    p->chains = chains;
    for (int i = 0; i < p->max_jobs; ++i) {  // admitted streaming jobs take the new chunking too
        JobDesc &D = p->h_jobs[i];
        if (!p->slots[i].live || D.resident) continue;
        D.nw = pool_words(D.geo, max_words);
        const FastDiv fdC = make_fastdiv((uint32_t)(D.geo.W / D.nw));
        D.divC_m = fdC.m;
        D.divC_l = fdC.l;
    }
    p->tables_dirty = true;
    return MICSA_OK;
}

}  // extern "C"
