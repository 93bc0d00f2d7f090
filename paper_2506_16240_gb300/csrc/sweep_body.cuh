// sweep_body.cuh -- the update of one thread's chunk of a row: the body shared
// by the single-handle half-sweep kernel and the batched (pool) kernel.
#pragma once

#include <type_traits>

#include "micsa_internal.h"

namespace micsa {

// Update NW words (4 NW sites) of row `row` (= z L + y) of parity p of one
// replica: spins/daemons point at that replica's [2][half] block, bonds at the
// sample's [2][half] block. gid is the replica's global id in the Philox
// counter, t the global sweep index. refresh: draw the daemon words instead of
// reading them (Sec. 2.7); METRO: Metropolis acceptance with the cut points th*.
// Read-only word loads from global (through the read-only path) or shared memory.
template <int NW, bool SMEM>
__device__ __forceinline__ void load_ro(const void *p, uint32_t (&w)[NW]) {
    if constexpr (SMEM) load_words<NW>(p, w);
    else load_words_ro<NW>(p, w);
}

template <bool SMEM>
__device__ __forceinline__ uint32_t load_byte(const int8_t *p) {
    if constexpr (SMEM) return (uint8_t)*p;
    else return (uint8_t)__ldg(p);
}

// FULL: rows without padding (P == Lh, so every lane is a site and a range of
// 4 NW bytes that reaches the row's end ends exactly at its last site).
template <int NW, bool METRO, bool SMEM = false, bool FULL = false>
__device__ __forceinline__ void update_chunk(const Geometry &g, int8_t *spins, uint8_t *daemons,
                                             const uint8_t *bonds, int p, int row, int c,
                                             uint32_t gid, uint32_t key0, uint32_t key1, int64_t t,
                                             bool refresh, uint64_t th0, uint64_t th1,
                                             uint64_t th2, const FastDiv &divL) {
    const int z = (int)fdiv((uint32_t)row, divL), y = row - z * g.L;
    const int o = (p + y + z) & 1;
    const int b0 = c * 4 * NW;  // first byte of this thread's range within the row
    const int yp = (y + 1 == g.L) ? 0 : y + 1, ym = (y == 0) ? g.L - 1 : y - 1;
    const int zp = (z + 1 == g.L) ? 0 : z + 1, zm = (z == 0) ? g.L - 1 : z - 1;
    // offsets within one parity half: 32-bit for MicSA (L^2 P < 2^32 bytes for
    // every allowed L; fewer instructions), 64-bit for the Metropolis variant
    // (measured faster there)
    using Off = typename std::conditional<METRO, int64_t, uint32_t>::type;
    const Off P = (Off)g.P, uL = (Off)g.L;
    const Off row0 = (Off)row * P;
    const Off off_c = row0 + (Off)b0;
    const int8_t *__restrict__ opp = spins + (int64_t)(1 - p) * g.half;
    int8_t *__restrict__ own_s = spins + (int64_t)p * g.half;
    uint8_t *__restrict__ own_d = daemons + (int64_t)p * g.half;

    uint32_t Bw[NW], O[NW], Oyp[NW], Oym[NW], Ozp[NW], Ozm[NW], S[NW], D[NW];
    load_ro<NW, SMEM>(bonds + (int64_t)p * g.half + off_c, Bw);
    load_ro<NW, SMEM>(opp + off_c, O);
    load_ro<NW, SMEM>(opp + (((Off)z * uL + (Off)yp) * P + (Off)b0), Oyp);
    load_ro<NW, SMEM>(opp + (((Off)z * uL + (Off)ym) * P + (Off)b0), Oym);
    load_ro<NW, SMEM>(opp + (((Off)zp * uL + (Off)y) * P + (Off)b0), Ozp);
    load_ro<NW, SMEM>(opp + (((Off)zm * uL + (Off)y) * P + (Off)b0), Ozm);
    load_words<NW>(own_s + off_c, S);
    if (!METRO && !refresh) load_words<NW>(own_d + off_c, D);

    // edge bytes for the x shift and the periodic wrap of the row
    uint32_t edge = 0, first = 0, last = 0;
    if constexpr (FULL) {
        // o = 0: the byte before the range, or the row's last byte at the row's start
        // o = 1: the byte after the range, or the row's first byte at the row's end
        // selected as an offset within the parity half: one pointer add, not four
        const Off eo = o == 0 ? (b0 == 0 ? row0 + (Off)(g.Lh - 1) : off_c - 1)
                              : (b0 + 4 * NW < g.Lh ? off_c + (Off)(4 * NW) : row0);
        edge = last = load_byte<SMEM>(opp + eo);
    } else if (o == 0) {
        if (b0 == 0) last = load_byte<SMEM>(opp + row0 + g.Lh - 1);
        else edge = load_byte<SMEM>(opp + off_c - 1);
    } else {
        if (b0 + 4 * NW <= g.Lh - 1) edge = load_byte<SMEM>(opp + off_c + 4 * NW);
        else first = (b0 == 0) ? (O[0] & 0xFFu) : load_byte<SMEM>(opp + row0);
    }
    uint32_t xp[NW], xm[NW];
    x_neighbours<NW, !FULL>(O, o, b0, g.Lh, edge, first, last, xp, xm);
    const uint32_t quad0 = (uint32_t)((((int64_t)p * g.L + z) * g.L + y) * g.W + c * NW);
    const RoundKeys rk = round_keys(key0, key1);  // invariant over the thread's chunks

#pragma unroll
    for (int j = 0; j < NW; ++j) {
        const uint32_t u32 = unsatisfied_count(Bw[j], S[j], xp[j], xm[j], Oyp[j], Oym[j], Ozp[j], Ozm[j]);
        const uint32_t valid = FULL ? 0xFFFFFFFFu : valid_mask(b0, j, g.Lh);
        if (METRO) {
            // dH = 12 - 4u > 0 <=> u < 3; accept iff a fresh uniform is below
            // the Metropolis cut point of dH (index 2 - u).
            const uint4 w = philox_wide(
                make_uint4(quad0 + j, (uint32_t)t, (gid << 2) | kTagMetro, (uint32_t)((uint64_t)t >> 32)), rk);
            uint32_t am = 0;
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const uint32_t u = (u32 >> (8 * l + 5)) & 7u;
                bool acc = u >= 3;
                if (!acc) {
                    const uint64_t cut = (u == 2) ? th0 : (u == 1) ? th1 : th2;
                    acc = (uint64_t)lane_of(w, l) < cut;
                }
                if (acc) am |= 0xFFu << (8 * l);
            }
            am &= valid;
            S[j] ^= am & 0xFEFEFEFEu;
        } else {
            if (refresh) {
                const uint4 w = philox_wide(
                    make_uint4(quad0 + j, (uint32_t)t, (gid << 2) | kTagDaemon, (uint32_t)((uint64_t)t >> 32)), rk);
                D[j] = (daemon_from_uniform(w.x, th0, th1, th2) |
                        (daemon_from_uniform(w.y, th0, th1, th2) << 8) |
                        (daemon_from_uniform(w.z, th0, th1, th2) << 16) |
                        (daemon_from_uniform(w.w, th0, th1, th2) << 24)) & valid;
            }
            const uint32_t am = creutz4(u32, D[j], valid);
            S[j] ^= am & 0xFEFEFEFEu;
        }
    }
    store_words<NW>(own_s + off_c, S);
    if (!METRO) store_words<NW>(own_d + off_c, D);
}

// Sum over the valid lanes of word w of an even row of (2u - 6): the energy of
// the bonds of those even sites (each bond has exactly one even end for even
// L, so the sum over all even words is H_EA). `even`/`odd` point at the two
// parity halves of one replica, `bonds` at the even bond half.
template <bool SMEM>
__device__ __forceinline__ int even_word_energy(const Geometry &g, const int8_t *even, const int8_t *odd,
                                                const uint8_t *bonds, int64_t w) {
    const int row = (int)(w / g.W);
    const int b0 = (int)(w - (int64_t)row * g.W) * 4;
    const int y = row % g.L, z = row / g.L;
    const int o = (y + z) & 1;
    const int yp = (y + 1 == g.L) ? 0 : y + 1, ym = (y == 0) ? g.L - 1 : y - 1;
    const int zp = (z + 1 == g.L) ? 0 : z + 1, zm = (z == 0) ? g.L - 1 : z - 1;
    const int64_t row0 = (int64_t)row * g.P, off = row0 + b0;
    const uint32_t valid = valid_mask(b0, 0, g.Lh);
    uint32_t O[1], Oyp[1], Oym[1], Ozp[1], Ozm[1], B[1], S[1];
    load_ro<1, SMEM>(odd + off, O);
    load_ro<1, SMEM>(odd + ((int64_t)z * g.L + yp) * g.P + b0, Oyp);
    load_ro<1, SMEM>(odd + ((int64_t)z * g.L + ym) * g.P + b0, Oym);
    load_ro<1, SMEM>(odd + ((int64_t)zp * g.L + y) * g.P + b0, Ozp);
    load_ro<1, SMEM>(odd + ((int64_t)zm * g.L + y) * g.P + b0, Ozm);
    load_ro<1, SMEM>(bonds + off, B);
    load_ro<1, SMEM>(even + off, S);
    uint32_t edge = 0, first = 0, last = 0;
    if (o == 0) {
        if (b0 == 0) last = load_byte<SMEM>(odd + row0 + g.Lh - 1);
        else edge = load_byte<SMEM>(odd + off - 1);
    } else {
        if (b0 + 4 <= g.Lh - 1) edge = load_byte<SMEM>(odd + off + 4);
        else first = (b0 == 0) ? (O[0] & 0xFFu) : load_byte<SMEM>(odd + row0);
    }
    uint32_t xp[1], xm[1];
    x_neighbours<1>(O, o, b0, g.Lh, edge, first, last, xp, xm);
    const uint32_t u32 =
        unsatisfied_count(B[0], S[0], xp[0], xm[0], Oyp[0], Oym[0], Ozp[0], Ozm[0]) & valid;
    return 2 * (int)(((u32 >> 5) * 0x01010101u) >> 24) - 6 * (__popc(valid) / 8);
}

}  // namespace micsa

namespace micsa {

// The MicSA update of rows (z, y0) and (z, y0 + 1), y0 even, of parity p over
// the same NW words, for rows without padding (P == Lh). Both rows read the
// opposite-parity rows y0 and y0 + 1 (one as its own row, the other as its
// y neighbour), so the pair loads 8 opposite-parity words of NW instead of
// 10, and the row decode, addressing and loop overhead are shared.
template <int NW>
__device__ __forceinline__ void micsa_cells(const Geometry &g, uint32_t (&S)[NW], uint32_t (&D)[NW],
                                            const uint32_t (&Bw)[NW], const uint32_t (&O)[NW],
                                            const uint32_t (&Oyp)[NW], const uint32_t (&Oym)[NW],
                                            const uint32_t (&Ozp)[NW], const uint32_t (&Ozm)[NW], int o,
                                            uint32_t edge, uint32_t quad0, uint32_t gid, uint32_t key0,
                                            uint32_t key1, int64_t t, bool refresh, uint64_t th0, uint64_t th1,
                                            uint64_t th2) {
    uint32_t xp[NW], xm[NW];
    x_neighbours<NW, false>(O, o, 0, g.Lh, edge, 0u, edge, xp, xm);
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        if (refresh) {
            const uint4 w = philox4x32_10(
                make_uint4(quad0 + j, (uint32_t)t, (gid << 2) | kTagDaemon, (uint32_t)((uint64_t)t >> 32)), key0,
                key1);
            D[j] = daemon_from_uniform(w.x, th0, th1, th2) | (daemon_from_uniform(w.y, th0, th1, th2) << 8) |
                   (daemon_from_uniform(w.z, th0, th1, th2) << 16) | (daemon_from_uniform(w.w, th0, th1, th2) << 24);
        }
        const uint32_t am = creutz4(unsatisfied_count(Bw[j], S[j], xp[j], xm[j], Oyp[j], Oym[j], Ozp[j], Ozm[j]),
                                    D[j], 0xFFFFFFFFu);
        S[j] ^= am & 0xFEFEFEFEu;
    }
}

template <int NW>
__device__ __forceinline__ void update_pair(const Geometry &g, int8_t *spins, uint8_t *daemons,
                                            const uint8_t *bonds, int p, int z, int y0, int c, uint32_t gid,
                                            uint32_t key0, uint32_t key1, int64_t t, bool refresh, uint64_t th0,
                                            uint64_t th1, uint64_t th2) {
    const int L = g.L, P = g.P;
    const int b0 = c * 4 * NW;
    const int y1 = y0 + 1;
    const int ym = (y0 == 0) ? L - 1 : y0 - 1, y2 = (y1 + 1 == L) ? 0 : y1 + 1;
    const int zp = (z + 1 == L) ? 0 : z + 1, zm = (z == 0) ? L - 1 : z - 1;
    const int8_t *__restrict__ opp = spins + (int64_t)(1 - p) * g.half;
    int8_t *__restrict__ own_s = spins + (int64_t)p * g.half;
    uint8_t *__restrict__ own_d = daemons + (int64_t)p * g.half;
    const uint8_t *__restrict__ bnd = bonds + (int64_t)p * g.half;
    const int64_t r0 = ((int64_t)z * L + y0) * P, r1 = r0 + P;  // rows (z, y0), (z, y0 + 1)

    uint32_t A[NW], Bq[NW], C[NW], Dq[NW], Zp0[NW], Zm0[NW], Zp1[NW], Zm1[NW];
    load_words_ro<NW>(opp + ((int64_t)z * L + ym) * P + b0, A);
    load_words_ro<NW>(opp + r0 + b0, Bq);
    load_words_ro<NW>(opp + r1 + b0, C);
    load_words_ro<NW>(opp + ((int64_t)z * L + y2) * P + b0, Dq);
    load_words_ro<NW>(opp + ((int64_t)zp * L + y0) * P + b0, Zp0);
    load_words_ro<NW>(opp + ((int64_t)zm * L + y0) * P + b0, Zm0);
    load_words_ro<NW>(opp + ((int64_t)zp * L + y1) * P + b0, Zp1);
    load_words_ro<NW>(opp + ((int64_t)zm * L + y1) * P + b0, Zm1);
    uint32_t B0[NW], B1[NW], S0[NW], S1[NW], D0[NW], D1[NW];
    load_words_ro<NW>(bnd + r0 + b0, B0);
    load_words_ro<NW>(bnd + r1 + b0, B1);
    load_words<NW>(own_s + r0 + b0, S0);
    load_words<NW>(own_s + r1 + b0, S1);
    if (!refresh) {
        load_words<NW>(own_d + r0 + b0, D0);
        load_words<NW>(own_d + r1 + b0, D1);
    }
    // edge bytes: for x offset 0 the byte before the range (the row's last byte
    // at the row's start), for offset 1 the byte after it (the row's first byte
    // at the row's end); rows y0 and y0 + 1 have opposite offsets
    const int o0 = (p + y0 + z) & 1;
    const int before = b0 == 0 ? g.Lh - 1 : b0 - 1, after = b0 + 4 * NW < g.Lh ? b0 + 4 * NW : 0;
    const uint32_t e0 = (uint8_t)__ldg(opp + r0 + (o0 == 0 ? before : after));
    const uint32_t e1 = (uint8_t)__ldg(opp + r1 + (o0 == 0 ? after : before));
    const uint32_t quad0 = (uint32_t)((((int64_t)p * L + z) * L + y0) * g.W + c * NW);
    // x_neighbours with range start 0: the wrap is carried by the edge byte (rows without padding)
    micsa_cells<NW>(g, S0, D0, B0, Bq, C, A, Zp0, Zm0, o0, e0, quad0, gid, key0, key1, t, refresh, th0, th1, th2);
    micsa_cells<NW>(g, S1, D1, B1, C, Dq, Bq, Zp1, Zm1, 1 - o0, e1, quad0 + (uint32_t)g.W, gid, key0, key1, t,
                    refresh, th0, th1, th2);
    store_words<NW>(own_s + r0 + b0, S0);
    store_words<NW>(own_d + r0 + b0, D0);
    store_words<NW>(own_s + r1 + b0, S1);
    store_words<NW>(own_d + r1 + b0, D1);
}

// The MicSA update of one chunk (NW words of row `row`, parity p) for the
// replicas [0, nrep) of one sample in one thread, rows without padding: the
// bond words, the row decode and the neighbour offsets are computed once and
// shared by the replicas. spins / daemons point at replica 0's [2][half] block
// (daemon family of the sweep already applied), rep_stride bytes between
// consecutive replicas' blocks; fam0 is replica 0's Philox id, fam_step the
// step between replicas' ids.
template <int NW>
__device__ __forceinline__ void update_reps(const Geometry &g, int8_t *spins, uint8_t *daemons, int64_t rep_stride,
                                            int64_t drep_stride, const uint8_t *bonds, int p, int row, int c,
                                            int nrep, uint32_t fam0, uint32_t fam_step, uint32_t key0,
                                            uint32_t key1, int64_t t, bool refresh, uint64_t th0, uint64_t th1,
                                            uint64_t th2, const FastDiv &divL) {
    const int z = (int)fdiv((uint32_t)row, divL), y = row - z * g.L;
    const int o = (p + y + z) & 1;
    const int b0 = c * 4 * NW;
    const int yp = (y + 1 == g.L) ? 0 : y + 1, ym = (y == 0) ? g.L - 1 : y - 1;
    const int zp = (z + 1 == g.L) ? 0 : z + 1, zm = (z == 0) ? g.L - 1 : z - 1;
    const uint32_t P = (uint32_t)g.P, uL = (uint32_t)g.L;
    const uint32_t row0 = (uint32_t)row * P;
    const uint32_t off_c = row0 + (uint32_t)b0;
    const uint32_t off_yp = ((uint32_t)z * uL + (uint32_t)yp) * P + (uint32_t)b0;
    const uint32_t off_ym = ((uint32_t)z * uL + (uint32_t)ym) * P + (uint32_t)b0;
    const uint32_t off_zp = ((uint32_t)zp * uL + (uint32_t)y) * P + (uint32_t)b0;
    const uint32_t off_zm = ((uint32_t)zm * uL + (uint32_t)y) * P + (uint32_t)b0;
    // the edge byte of the x shift: before the range (offset 0) or after it (offset 1),
    // the row's other end at its ends
    const uint32_t eo = o == 0 ? (b0 == 0 ? row0 + (uint32_t)(g.Lh - 1) : off_c - 1)
                               : (b0 + 4 * NW < g.Lh ? off_c + (uint32_t)(4 * NW) : row0);
    uint32_t Bw[NW];
    load_words_ro<NW>(bonds + (int64_t)p * g.half + off_c, Bw);
    const uint32_t quad0 = (uint32_t)((((int64_t)p * g.L + z) * g.L + y) * g.W + c * NW);
    for (int r = 0; r < nrep; ++r) {
        const int8_t *__restrict__ opp = spins + r * rep_stride + (int64_t)(1 - p) * g.half;
        int8_t *__restrict__ own_s = spins + r * rep_stride + (int64_t)p * g.half;
        uint8_t *__restrict__ own_d = daemons + r * drep_stride + (int64_t)p * g.half;
        uint32_t O[NW], Oyp[NW], Oym[NW], Ozp[NW], Ozm[NW], S[NW], D[NW];
        load_words_ro<NW>(opp + off_c, O);
        load_words_ro<NW>(opp + off_yp, Oyp);
        load_words_ro<NW>(opp + off_ym, Oym);
        load_words_ro<NW>(opp + off_zp, Ozp);
        load_words_ro<NW>(opp + off_zm, Ozm);
        load_words<NW>(own_s + off_c, S);
        if (!refresh) load_words<NW>(own_d + off_c, D);
        const uint32_t edge = (uint8_t)__ldg(opp + eo);
        micsa_cells<NW>(g, S, D, Bw, O, Oyp, Oym, Ozp, Ozm, o, edge, quad0, fam0 + (uint32_t)r * fam_step, key0,
                        key1, t, refresh, th0, th1, th2);
        store_words<NW>(own_s + off_c, S);
        store_words<NW>(own_d + off_c, D);
    }
}

}  // namespace micsa
