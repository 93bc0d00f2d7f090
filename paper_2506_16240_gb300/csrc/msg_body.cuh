// msg_body.cuh -- the bit-plane (multispin-coded) half-sweep of one thread:
// the body shared by the single-handle bit-plane kernel and the batched
// (pool) kernel, and the helpers of the shared-memory multispin kernel.
#pragma once

#include "micsa_internal.h"

namespace micsa {

// Refresh cut points as strict 32-bit compares: [u >= c] = [u > c - 1]. Valid
// for 1 <= c <= 2^32; every cut point is >= floor(2^32 p(0)) >= 2^30, since
// p(0) = 1 / (1 + x + x^2 + x^3) >= 1/4 for x = exp(-4 beta) <= 1. With the
// cut points increasing, m = [u >= c0] + [u >= c1] + [u >= c2] has bit 1 =
// [u >= c1] and bit 0 = the parity of the three.
struct CutsGt {
    uint32_t c0m, c1m, c2m;
};

__device__ __forceinline__ CutsGt make_cuts_gt(uint64_t th0, uint64_t th1, uint64_t th2) {
    return {(uint32_t)(th0 - 1), (uint32_t)(th1 - 1), (uint32_t)(th2 - 1)};
}

// x_k = 2 x_k + [u > c_k] for three cut points given as n_k = ~c_k: the carry
// out of u + ~c is set exactly when u > c, and addc shifts it in.
__device__ __forceinline__ void shift_in_cuts(uint32_t u, uint32_t n0, uint32_t n1, uint32_t n2, uint32_t &x0,
                                              uint32_t &x1, uint32_t &x2) {
    asm("{\n\t.reg .u32 t;\n\t"
        "add.cc.u32 t, %3, %4;\n\taddc.u32 %0, %0, %0;\n\t"
        "add.cc.u32 t, %3, %5;\n\taddc.u32 %1, %1, %1;\n\t"
        "add.cc.u32 t, %3, %6;\n\taddc.u32 %2, %2, %2;\n\t}"
        : "+r"(x0), "+r"(x1), "+r"(x2)
        : "r"(u), "r"(n0), "r"(n1), "r"(n2));
}

// x_k = 2 x_k + [u < t_k] for three Metropolis cut points: the carry out of
// t_k + ~u is set exactly when t_k > u.
__device__ __forceinline__ void shift_in_below(uint32_t u, uint32_t t0, uint32_t t1, uint32_t t2, uint32_t &x0,
                                               uint32_t &x1, uint32_t &x2) {
    const uint32_t nu = ~u;
    asm("{\n\t.reg .u32 t;\n\t"
        "add.cc.u32 t, %3, %6;\n\taddc.u32 %0, %0, %0;\n\t"
        "add.cc.u32 t, %4, %6;\n\taddc.u32 %1, %1, %1;\n\t"
        "add.cc.u32 t, %5, %6;\n\taddc.u32 %2, %2, %2;\n\t}"
        : "+r"(x0), "+r"(x1), "+r"(x2)
        : "r"(t0), "r"(t1), "r"(t2), "r"(nu));
}

__device__ __forceinline__ void prefetch_l2(const uint32_t *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <int NW> struct Vec;
template <> struct Vec<1> {
    static __device__ __forceinline__ void ld(const uint32_t *p, uint32_t *v) { v[0] = *p; }
    static __device__ __forceinline__ void st(uint32_t *p, const uint32_t *v) { *p = v[0]; }
};
template <> struct Vec<2> {
    static __device__ __forceinline__ void ld(const uint32_t *p, uint32_t *v) {
        const uint2 a = *reinterpret_cast<const uint2 *>(p);
        v[0] = a.x;
        v[1] = a.y;
    }
    static __device__ __forceinline__ void st(uint32_t *p, const uint32_t *v) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(v[0], v[1]);
    }
};
template <> struct Vec<4> {
    static __device__ __forceinline__ void ld(const uint32_t *p, uint32_t *v) {
        const uint4 a = *reinterpret_cast<const uint4 *>(p);
        v[0] = a.x;
        v[1] = a.y;
        v[2] = a.z;
        v[3] = a.w;
    }
    static __device__ __forceinline__ void st(uint32_t *p, const uint32_t *v) {
        *reinterpret_cast<uint4 *>(p) = make_uint4(v[0], v[1], v[2], v[3]);
    }
};

// Daemon words of the NW own words after a wandering step along direction dd
// (0 +x, 1 +y, 2 +z, 3 -x, 4 -y, 5 -z): the words of the other parity's plane
// Sx at that neighbour, assembled like the spin neighbours of the update (M:
// bits whose own site has x offset 1; w_*: the neighbour word indices).
template <int NW>
__device__ __forceinline__ void gather_words(const uint32_t *Sx, int dd, int64_t wc, int64_t w_ip, int64_t w_im,
                                             int64_t w_yp, int64_t w_ym, int64_t w_zp, int64_t w_zm, uint32_t M,
                                             uint32_t (&out)[NW]) {
    uint32_t c[NW], n[NW];
    Vec<NW>::ld(Sx + wc, c);
    if (dd == 0 || dd == 3) {
        const uint32_t edge = Sx[dd == 0 ? w_ip : w_im];
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            if (dd == 0) {
                const uint32_t nx = w + 1 < NW ? c[w + 1 < NW ? w + 1 : 0] : edge;
                out[w] = (c[w] & ~M) | (nx & M);
            } else {
                const uint32_t pv = w > 0 ? c[w > 0 ? w - 1 : 0] : edge;
                out[w] = (pv & ~M) | (c[w] & M);
            }
        }
        return;
    }
    const int64_t wn = dd == 1 ? w_yp : dd == 4 ? w_ym : dd == 2 ? w_zp : w_zm;
    Vec<NW>::ld(Sx + wn, n);
#pragma unroll
    for (int w = 0; w < NW; ++w)
        out[w] = dd == 1 || dd == 4 ? n[w] : dd == 2 ? __funnelshift_r(c[w], n[w], 1) : __funnelshift_l(n[w], c[w], 1);
}

// One sample's bit planes as a half-sweep thread sees them: replica r's planes
// start at planes + r * np * WP; the sample's bond planes are [6][2][WP].
struct MsgLattice {
    uint32_t *planes;
    const uint32_t *bonds;
    int L, Lh, nzw, W4;  // Lh: plane words per row (the row stride); W4 = Lh / 4 Philox blocks per row
    int64_t WP;
    int np, gamma, walkers;  // planes per replica, daemon families, two daemon buffers
    int64_t gid0;            // Philox id of replica 0 (sample * R)
    uint32_t key0, key1;
    int Lr;  // sites per row of one parity, L / 2; below Lh when the row is padded to whole Philox blocks
};

// Plane word w of parity p of replica rep <-> the 32 sites of its z column in
// the byte layout (spins, and the gamma daemon families of buffer buf).
__device__ __forceinline__ void msg_convert_word(uint32_t *planes, int8_t *spins, uint8_t *daemons, const Geometry &g,
                                                 int64_t WP, int gamma, int np, int buf, bool to_planes, int64_t rep,
                                                 int p, int64_t w) {
    // rows of g.P plane words (the byte layout's pitch, whole Philox blocks); the
    // words from g.Lh on hold no site and stay zero in the planes
    const int i = (int)(w % g.P);
    const int y = (int)((w / g.P) % g.L);
    const int zw = (int)(w / ((int64_t)g.P * g.L));
    const int64_t in_half = ((int64_t)32 * zw * g.L + y) * g.P + i;
    const int64_t zstep = (int64_t)g.L * g.P;
    uint32_t *pl = planes + rep * np * WP;
    if (i >= g.Lh) {
        if (to_planes) {
            pl[(int64_t)p * WP + w] = 0;
            for (int al = 0; al < gamma; ++al) {
                const int mp = 2 + ((buf * gamma + al) * 2) * 2 + p;
                pl[(int64_t)mp * WP + w] = 0;
                pl[(int64_t)(mp + 2) * WP + w] = 0;
            }
        }
        return;
    }
    const int64_t sbase = (rep * 2 + p) * g.half + in_half;
    const int nb = g.L - 32 * zw < 32 ? g.L - 32 * zw : 32;  // sites of the column in this word
    if (to_planes) {
        uint32_t sv = 0;
        for (int b = 0; b < nb; ++b) sv |= (((uint32_t)(uint8_t)spins[sbase + b * zstep] >> 7) & 1u) << b;
        pl[(int64_t)p * WP + w] = sv;
    } else {
        const uint32_t sv = pl[(int64_t)p * WP + w];
        for (int b = 0; b < nb; ++b) spins[sbase + b * zstep] = ((sv >> b) & 1u) ? (int8_t)-1 : (int8_t)1;
    }
    for (int al = 0; al < gamma; ++al) {
        const int64_t dbase = ((rep * gamma + al) * 2 + p) * g.half + in_half;
        const int mp = 2 + ((buf * gamma + al) * 2) * 2 + p;
        if (to_planes) {
            uint32_t m0 = 0, m1 = 0;
            for (int b = 0; b < nb; ++b) {
                const uint32_t m = daemons[dbase + b * zstep];
                m0 |= (m & 1u) << b;
                m1 |= ((m >> 1) & 1u) << b;
            }
            pl[(int64_t)mp * WP + w] = m0;
            pl[(int64_t)(mp + 2) * WP + w] = m1;
        } else {
            const uint32_t m0 = pl[(int64_t)mp * WP + w], m1 = pl[(int64_t)(mp + 2) * WP + w];
            for (int b = 0; b < nb; ++b)
                daemons[dbase + b * zstep] = (uint8_t)(((m0 >> b) & 1u) | (((m1 >> b) & 1u) << 1));
        }
    }
}

// One thread's half-sweep (parity p) of the NW plane words (32 NW sites) at
// (zw, y, NW * ig) of lattice a, for its replicas [r_begin, r_end): Eq. (Creutz)
// with Eq. (flip-OK) on 32 sites per word, bit-sliced; at a refresh sweep the
// daemons are drawn first (Sec. 2.7), with walkers the previous wandering step
// is applied on read (Sec. 2.6). Lanes (threadIdx.x & (4 / NW - 1)) share one
// Philox block, so the threads of a warp must all be active. RAGGED: the last
// word of a z column holds Lz = L - 32 (nzw - 1) sites (any even L > 32; no
// walkers): the z wrap goes through bit Lz - 1 of that word, and its
// bits from Lz up stay zero. METRO: the Metropolis sweep on the same planes
// (the daemon planes are neither read nor written). PREFETCH: the next
// replica's words are prefetched into L2 (planes in global memory only; a
// caller whose planes live in shared memory passes false).
// PADDED: rows of a.Lh words hold a.Lr < a.Lh sites (the words from a.Lr on
// are padding: never flipped, never a neighbour of a site; the +x wrap of the
// row's last site comes from word 0).
template <int NW, bool RAGGED = false, bool METRO = false, bool PREFETCH = true, bool PADDED = false>
__device__ __forceinline__ void msg_update(const MsgLattice &a, const SweepParam &prm, int p, int zw, int y, int ig,
                                           int r_begin, int r_end) {
    constexpr int G = 4 / NW;  // lanes sharing one Philox block of words
    const bool refresh = prm.mode == kModeRefresh;
    constexpr bool metro = METRO;  // Metropolis sweeps (one daemon family, no walkers)
    const int o = 1 - p;
    const int L = a.L, Lh = a.Lh;
    const int Lr = PADDED ? a.Lr : Lh;  // sites per row
    const int i0 = NW * ig;
    const int yp = (y + 1 == L) ? 0 : y + 1, ym = (y == 0) ? L - 1 : y - 1;
    const int zwp = (zw + 1 == a.nzw) ? 0 : zw + 1, zwm = (zw == 0) ? a.nzw - 1 : zw - 1;
    const int ip = (i0 + NW >= Lr) ? 0 : i0 + NW, im = (i0 == 0) ? Lr - 1 : i0 - 1;
    const int64_t row = (int64_t)zw * L;
    const int64_t wc = (row + y) * Lh + i0;
    const int64_t w_yp = (row + yp) * Lh + i0, w_ym = (row + ym) * Lh + i0;
    const int64_t w_zp = ((int64_t)zwp * L + y) * Lh + i0, w_zm = ((int64_t)zwm * L + y) * Lh + i0;
    const int64_t w_ip = (row + y) * Lh + ip, w_im = (row + y) * Lh + im;
    const uint32_t M = ((p + y) & 1) ? 0x55555555u : 0xAAAAAAAAu;  // bits whose site has x offset 1
    const int Lz = RAGGED ? L - 32 * (a.nzw - 1) : 32;  // sites in the last word of a column
    const uint32_t zmask = (RAGGED && zw == a.nzw - 1 && Lz < 32) ? ((1u << Lz) - 1u) : 0xFFFFFFFFu;

    uint32_t B[6][NW];
    const uint32_t *bs = a.bonds;
#pragma unroll
    for (int k = 0; k < 6; ++k) Vec<NW>::ld(bs + ((int64_t)k * 2 + p) * a.WP + wc, B[k]);
    const RoundKeys rk = round_keys(a.key0, a.key1);
    const CutsGt gcut = make_cuts_gt(prm.th0, prm.th1, prm.th2);
    const int lig = (int)(threadIdx.x & (G - 1));  // this lane's share of the Philox block
    const uint32_t quad0 = (uint32_t)(((int64_t)p * L + 32 * zw) * L + y) * a.W4 + (uint32_t)(i0 >> 2);

    const int alpha = prm.alpha, buf = a.walkers ? (int)(prm.t & 1) : 0;
    const int mplane = 2 + ((buf * a.gamma + alpha) * 2) * 2 + p;  // m0 of (buffer, family, parity p)
    const bool gather = prm.gather != 0 && !refresh;
    // gather source: m0 of (the other buffer, family, the other parity); the direction of the
    // previous wandering step seen from parity p
    const int gplane = 2 + (((1 - buf) * a.gamma + alpha) * 2) * 2 + o;
    const int gq = (int)((prm.t - 1) & 1), gd0 = alpha % 6, gdd = (p == gq) ? gd0 : (gd0 + 3) % 6;
    const int mread = gather ? gplane : mplane;  // the daemon words this half-sweep reads
    for (int r = r_begin; r < r_end; ++r) {
        const int64_t gid = a.gid0 + r;
        const uint32_t fam = (uint32_t)(gid * a.gamma + alpha);  // Philox id of this daemon family
        uint32_t *pl = a.planes + (int64_t)r * a.np * a.WP;
        if (PREFETCH && r + 1 < r_end) {  // the next replica's words that come from DRAM, into L2
            const uint32_t *nx = pl + (int64_t)a.np * a.WP;
            prefetch_l2(nx + (int64_t)p * a.WP + wc);
            prefetch_l2(nx + (int64_t)o * a.WP + wc);
            if (!refresh && !metro) {  // (a Metropolis sweep reads no daemon words)
                prefetch_l2(nx + (int64_t)mread * a.WP + wc);
                prefetch_l2(nx + (int64_t)(mread + 2) * a.WP + wc);
            }
        }
        const uint32_t *O = pl + (int64_t)o * a.WP;  // spins of the opposite parity
        uint32_t *Sp = pl + (int64_t)p * a.WP;
        uint32_t *M0 = pl + (int64_t)mplane * a.WP;
        uint32_t *M1 = pl + (int64_t)(mplane + 2) * a.WP;
        uint32_t Oc[NW], Oyp[NW], Oym[NW], Ozp[NW], Ozm[NW], Sg[NW], m0v[NW], m1v[NW];
        Vec<NW>::ld(O + wc, Oc);
        Vec<NW>::ld(O + w_yp, Oyp);
        Vec<NW>::ld(O + w_ym, Oym);
        Vec<NW>::ld(O + w_zp, Ozp);
        Vec<NW>::ld(O + w_zm, Ozm);
        const uint32_t Oip = O[w_ip], Oim = O[w_im];
        Vec<NW>::ld(Sp + wc, Sg);
        uint32_t a2v[NW];  // Metropolis: the acceptance bits of dH = 12 (of dH = 4, 8 in m0v, m1v)
        if (refresh) {  // fresh daemons of parity p before its half-sweep (Sec. 2.7)
            // z = 32 zw + b for b in this lane's range, from the top down: each new
            // bit enters at the bottom (a = 2 a + bit); m1 = [u >= c1], m0 = the parity
            // of [u >= c0] + [u >= c1] + [u >= c2]
            // x_k collects [u > c_k - 1] for the three cut points, one bit per z;
            // m0 = x_0 ^ x_1 ^ x_2 and m1 = x_1 (the cut points increase)
            uint32_t x0[4] = {0, 0, 0, 0}, a1[4] = {0, 0, 0, 0}, x2[4] = {0, 0, 0, 0};
            const uint32_t n0 = ~gcut.c0m, n1 = ~gcut.c1m, n2 = ~gcut.c2m;
#pragma unroll 2
            for (int c = 32 / G - 1; c >= 0; --c) {
                const int b = lig * (32 / G) + c;
                const uint4 w = philox_wide(make_uint4(quad0 + (uint32_t)b * (uint32_t)L * (uint32_t)a.W4, (uint32_t)prm.t,
                                                       (fam << 2) | kTagDaemon, (uint32_t)((uint64_t)prm.t >> 32)),
                                            rk);
                const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) shift_in_cuts(u[j], n0, n1, n2, x0[j], a1[j], x2[j]);
            }
            uint32_t a0[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                a0[j] = (x0[j] ^ a1[j] ^ x2[j]) << (lig * (32 / G));
                a1[j] <<= lig * (32 / G);
            }
#pragma unroll
            for (int off = 1; off < G; off <<= 1)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    a0[j] |= __shfl_xor_sync(0xFFFFFFFFu, a0[j], off);
                    a1[j] |= __shfl_xor_sync(0xFFFFFFFFu, a1[j], off);
                }
#pragma unroll
            for (int w = 0; w < NW; ++w) {  // word i0 + w is lane (i0 + w) & 3 of the block
                const int j = (i0 + w) & 3;
                const uint32_t wm = (!PADDED || i0 + w < Lr) ? zmask : 0u;  // padding words keep m = 0
                m0v[w] = (j == 0 ? a0[0] : j == 1 ? a0[1] : j == 2 ? a0[2] : a0[3]) & wm;
                m1v[w] = (j == 0 ? a1[0] : j == 1 ? a1[1] : j == 2 ? a1[2] : a1[3]) & wm;
            }
        } else if (metro) {
            // Metropolis (the canonical baseline of Sec. 2.4): one uniform per site from
            // the Philox block of its quad (lane i & 3, the Metropolis tag), z = 32 zw + b
            // from the top down; x_k collects [u < theta_k], the acceptance of dH =
            // 4 (k + 1), theta_k = 2^32 accepting every u. m0v, m1v, a2v take the planes.
            uint32_t x0[4] = {0, 0, 0, 0}, x1[4] = {0, 0, 0, 0}, x2[4] = {0, 0, 0, 0};
            const uint32_t mt0 = (uint32_t)prm.th0, mt1 = (uint32_t)prm.th1, mt2 = (uint32_t)prm.th2;
#pragma unroll 2
            for (int c = 32 / G - 1; c >= 0; --c) {
                const int b = lig * (32 / G) + c;
                const uint4 w = philox_wide(make_uint4(quad0 + (uint32_t)b * (uint32_t)L * (uint32_t)a.W4, (uint32_t)prm.t,
                                                       ((uint32_t)gid << 2) | kTagMetro, (uint32_t)((uint64_t)prm.t >> 32)),
                                            rk);
                const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) shift_in_below(u[j], mt0, mt1, mt2, x0[j], x1[j], x2[j]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                x0[j] = ((prm.th0 >> 32) ? ~0u : x0[j]) << (lig * (32 / G));
                x1[j] = ((prm.th1 >> 32) ? ~0u : x1[j]) << (lig * (32 / G));
                x2[j] = ((prm.th2 >> 32) ? ~0u : x2[j]) << (lig * (32 / G));
            }
#pragma unroll
            for (int off = 1; off < G; off <<= 1)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    x0[j] |= __shfl_xor_sync(0xFFFFFFFFu, x0[j], off);
                    x1[j] |= __shfl_xor_sync(0xFFFFFFFFu, x1[j], off);
                    x2[j] |= __shfl_xor_sync(0xFFFFFFFFu, x2[j], off);
                }
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const int j = (i0 + w) & 3;
                m0v[w] = (j == 0 ? x0[0] : j == 1 ? x0[1] : j == 2 ? x0[2] : x0[3]) & zmask;
                m1v[w] = (j == 0 ? x1[0] : j == 1 ? x1[1] : j == 2 ? x1[2] : x1[3]) & zmask;
                a2v[w] = (j == 0 ? x2[0] : j == 1 ? x2[1] : j == 2 ? x2[2] : x2[3]) & zmask;
            }
        } else if (gather) {  // the walkers arrive through the previous wandering step
            const uint32_t *G0 = pl + (int64_t)gplane * a.WP;
            gather_words<NW>(G0, gdd, wc, w_ip, w_im, w_yp, w_ym, w_zp, w_zm, M, m0v);
            gather_words<NW>(G0 + 2 * a.WP, gdd, wc, w_ip, w_im, w_yp, w_ym, w_zp, w_zm, M, m1v);
        } else {
            Vec<NW>::ld(M0 + wc, m0v);
            Vec<NW>::ld(M1 + wc, m1v);
        }
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t oc = Oc[w];
            uint32_t o_next = w + 1 < NW ? Oc[w + 1 < NW ? w + 1 : 0] : Oip;  // word i + 1
            if (PADDED && i0 + w + 1 == Lr) o_next = Oip;  // the row's last site wraps to word 0
            const uint32_t o_prev = w > 0 ? Oc[w > 0 ? w - 1 : 0] : Oim;            // word i - 1
            const uint32_t nxp = (oc & ~M) | (o_next & M);
            const uint32_t nxm = (o_prev & ~M) | (oc & M);
            uint32_t nzp = __funnelshift_r(oc, Ozp[w], 1);  // bit b <- site z + 1
            uint32_t nzm = __funnelshift_l(Ozm[w], oc, 1);  // bit b <- site z - 1
            if (RAGGED) {  // the wrap through a partial last word (the same bits when Lz == 32)
                if (zw == a.nzw - 1) nzp = (oc >> 1) | ((Ozp[w] & 1u) << (Lz - 1));
                if (zw == 0) nzm = (oc << 1) | ((Ozm[w] >> (Lz - 1)) & 1u);
            }
            const uint32_t sg = Sg[w];
            // unsatisfied bond indicators (J s s_nb = -1)
            const uint32_t q0 = sg ^ nxp ^ B[0][w];
            const uint32_t q1 = sg ^ Oyp[w] ^ B[1][w];
            const uint32_t q2 = sg ^ nzp ^ B[2][w];
            const uint32_t q3 = sg ^ nxm ^ B[3][w];
            const uint32_t q4 = sg ^ Oym[w] ^ B[4][w];
            const uint32_t q5 = sg ^ nzm ^ B[5][w];
            // u = q0 + ... + q5, then v = u + m, bit-sliced
            const uint32_t s1 = q0 ^ q1 ^ q2, c1 = (q0 & q1) | (q2 & (q0 ^ q1));
            const uint32_t s2 = q3 ^ q4 ^ q5, c2 = (q3 & q4) | (q5 & (q3 ^ q4));
            const uint32_t u0 = s1 ^ s2, kk = s1 & s2;
            const uint32_t u1 = c1 ^ c2 ^ kk, u2 = (c1 & c2) | (kk & (c1 ^ c2));
            const uint32_t m0 = m0v[w], m1 = m1v[w];
            uint32_t acc;
            if (metro) {
                // dH = 12 - 4u: accepted when dH <= 0 (u >= 3), else by the site's bit of dH
                const uint32_t nu2 = ~u2;
                acc = (u2 | (u1 & u0)) | (nu2 & u1 & ~u0 & m0) | (nu2 & ~u1 & u0 & m1) | (nu2 & ~u1 & ~u0 & a2v[w]);
                acc &= zmask;
            } else {
                const uint32_t v0 = u0 ^ m0, k0 = u0 & m0;
                const uint32_t v1 = u1 ^ m1 ^ k0, k1 = (u1 & m1) | (k0 & (u1 ^ m1));
                const uint32_t v2 = u2 ^ k1, v3 = u2 & k1;
                // Eq. (Creutz) with Eq. (flip-OK): accept <=> 3 <= u + m <= 6, m' = u + m - 3
                acc = (v2 ^ (v1 & v0)) & ~v3 & zmask;
                if (PADDED && i0 + w >= Lr) acc = 0;  // a padding word holds no site
                m0v[w] = (m0 & ~acc) | (~v0 & acc);
                m1v[w] = (m1 & ~acc) | (v2 & (v1 | v0) & acc);
            }
            Sg[w] = sg ^ acc;
        }
        Vec<NW>::st(Sp + wc, Sg);
        if (!metro) {
            Vec<NW>::st(M0 + wc, m0v);
            Vec<NW>::st(M1 + wc, m1v);
        }
    }
}


}  // namespace micsa
