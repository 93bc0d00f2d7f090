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
#include "micsa_internal.h"

namespace micsa {

template <int NW, int MODE>
__global__ void __launch_bounds__(256) half_sweep_kernel(SweepArgs a) {
    const Geometry g = a.geo;
    const int chunks = g.W / NW;
    const int64_t per_sample = (int64_t)g.L * g.L * chunks;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= per_sample * a.S) return;
    const int sample = (int)(tid / per_sample);
    const int64_t rem = tid - (int64_t)sample * per_sample;
    const int row = (int)(rem / chunks);
    const int c = (int)(rem - (int64_t)row * chunks);
    const int y = row % g.L, z = row / g.L;
    const int p = a.parity;
    const int o = (p + y + z) & 1;
    const int b0 = c * 4 * NW;  // first byte of this thread's range within the row

    const int yp = (y + 1 == g.L) ? 0 : y + 1, ym = (y == 0) ? g.L - 1 : y - 1;
    const int zp = (z + 1 == g.L) ? 0 : z + 1, zm = (z == 0) ? g.L - 1 : z - 1;
    const int64_t off_c = (int64_t)row * g.P + b0;
    const int64_t off_yp = ((int64_t)z * g.L + yp) * g.P + b0;
    const int64_t off_ym = ((int64_t)z * g.L + ym) * g.P + b0;
    const int64_t off_zp = ((int64_t)zp * g.L + y) * g.P + b0;
    const int64_t off_zm = ((int64_t)zm * g.L + y) * g.P + b0;
    const int64_t row0 = (int64_t)row * g.P;  // start of the row

    uint32_t Bw[NW];
    load_words<NW>(a.bonds + (int64_t)(sample * 2 + p) * g.half + off_c, Bw);

    const uint32_t quad0 = (uint32_t)((((int64_t)p * g.L + z) * g.L + y) * g.W + c * NW);

    for (int r = 0; r < a.R; ++r) {
        const int64_t gid = (int64_t)sample * a.R + r;
        const int8_t *opp = a.spins + (gid * 2 + (1 - p)) * g.half;
        int8_t *own_s = a.spins + (gid * 2 + p) * g.half;
        uint8_t *own_d = a.daemons + (gid * 2 + p) * g.half;

        uint32_t O[NW], Oyp[NW], Oym[NW], Ozp[NW], Ozm[NW], S[NW], D[NW];
        load_words_ro<NW>(opp + off_c, O);
        load_words_ro<NW>(opp + off_yp, Oyp);
        load_words_ro<NW>(opp + off_ym, Oym);
        load_words_ro<NW>(opp + off_zp, Ozp);
        load_words_ro<NW>(opp + off_zm, Ozm);
        load_words<NW>(own_s + off_c, S);
        if (MODE == kModeMicsa) load_words<NW>(own_d + off_c, D);

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

#pragma unroll
        for (int j = 0; j < NW; ++j) {
            const BondPlanes bp = bond_planes(Bw[j]);
            const uint32_t neg = negative_terms(bp, xp[j], xm[j], Oyp[j], Oym[j], Ozp[j], Ozm[j]);
            const uint32_t u32 = unsatisfied32(neg, S[j]);
            const uint32_t valid = valid_mask(b0, j, g.Lh);
            if (MODE == kModeMetro) {
                // dH = 12 - 4u > 0 <=> u < 3; accept iff a fresh uniform is below
                // the Metropolis cut point of dH (index 2 - u).
                const uint4 w = philox4x32_10(
                    make_uint4(quad0 + j, (uint32_t)a.t, (uint32_t)(gid << 2) | kTagMetro,
                               (uint32_t)((uint64_t)a.t >> 32)),
                    a.key0, a.key1);
                uint32_t am = 0;
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    const uint32_t u = (u32 >> (8 * l + 5)) & 7u;
                    bool acc = u >= 3;
                    if (!acc) {
                        const uint64_t cut = (u == 2) ? a.th0 : (u == 1) ? a.th1 : a.th2;
                        acc = (uint64_t)lane_of(w, l) < cut;
                    }
                    if (acc) am |= 0xFFu << (8 * l);
                }
                am &= valid;
                S[j] ^= am & 0xFEFEFEFEu;
            } else {
                if (MODE == kModeRefresh) {
                    const uint4 w = philox4x32_10(
                        make_uint4(quad0 + j, (uint32_t)a.t, (uint32_t)(gid << 2) | kTagDaemon,
                                   (uint32_t)((uint64_t)a.t >> 32)),
                        a.key0, a.key1);
                    D[j] = 0;
#pragma unroll
                    for (int l = 0; l < 4; ++l)
                        D[j] |= daemon_from_uniform(lane_of(w, l), a.th0, a.th1, a.th2) << (8 * l);
                    D[j] &= valid;
                }
                const uint32_t am = creutz4(u32, D[j], valid);
                S[j] ^= am & 0xFEFEFEFEu;
            }
        }
        store_words<NW>(own_s + off_c, S);
        if (MODE != kModeMetro) store_words<NW>(own_d + off_c, D);
    }
}

template <int MODE>
static cudaError_t launch_mode(const SweepArgs &a, cudaStream_t st) {
    const int nw = (a.geo.W % 4 == 0) ? 4 : 1;
    const int64_t threads = (int64_t)a.S * a.geo.L * a.geo.L * (a.geo.W / nw);
    const int block = 256;
    const int64_t grid = (threads + block - 1) / block;
    if (nw == 4)
        half_sweep_kernel<4, MODE><<<(unsigned)grid, block, 0, st>>>(a);
    else
        half_sweep_kernel<1, MODE><<<(unsigned)grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_half_sweep(const SweepArgs &a, int mode, cudaStream_t st) {
    switch (mode) {
        case kModeMicsa: return launch_mode<kModeMicsa>(a, st);
        case kModeRefresh: return launch_mode<kModeRefresh>(a, st);
        case kModeMetro: return launch_mode<kModeMetro>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace micsa
