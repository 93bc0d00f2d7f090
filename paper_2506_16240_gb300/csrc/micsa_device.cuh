// micsa_device.cuh -- device-side building blocks shared by the sweep,
// initialisation and measurement kernels.
//
// Device layout (sublattice split, Sec. 2.1): each (sample, replica) holds two
// parity halves; a half is L planes (z) x L rows (y) x P bytes, where row
// (z, y) of parity p stores the L/2 sites x = 2i + ((p + y + z) & 1),
// i = 0..L/2-1, at bytes 0..L/2-1 and zero padding up to the pitch
// P = 4 * ceil(L/2 / 4). Spins are int8 +-1 (0x01 / 0xFF), daemons uint8 m in
// {0..3}; a bond byte per site holds the six incident couplings, bit k set <=>
// J = -1 for k = 0: +x, 1: +y, 2: +z, 3: -x, 4: -y, 5: -z. Bonds are shared by
// the replicas of a sample.
//
// Four sites of a row travel together in one 32-bit word (byte lane i & 3).
// Bit 5 of a spin byte is its sign bit (0x01 -> 0, 0xFF -> 1), so the
// per-lane arithmetic below runs on all four lanes of a word at once.
#pragma once

#include <cstdint>

namespace micsa {

constexpr uint32_t kTagCoupling = 0, kTagSpin = 1, kTagDaemon = 2, kTagMetro = 3;

// ----------------------------------------------------------------- Philox --
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// two-multiplier S-box with the Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
    constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
    constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // high and low words of each 32 x 32 -> 64-bit product
        const uint64_t p0 = (uint64_t)kM0 * c.x, p1 = (uint64_t)kM1 * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
        k0 += kW0;
        k1 += kW1;
    }
    return c;
}

// Philox4x32-10 with the ten round keys precomputed (same function as
// philox4x32_10: round r uses key + r * Weyl increment).
struct RoundKeys {
    uint32_t k0[10], k1[10];
};

__device__ __forceinline__ RoundKeys round_keys(uint32_t key0, uint32_t key1) {
    RoundKeys r;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        r.k0[i] = key0 + (uint32_t)i * 0x9E3779B9u;
        r.k1[i] = key1 + (uint32_t)i * 0xBB67AE85u;
    }
    return r;
}

// Philox4x32-10 with the round keys precomputed, each round's two products
// taken as one 32 x 32 -> 64-bit multiply (high word and low word of the same
// product).
__device__ __forceinline__ uint4 philox_wide(uint4 c, const RoundKeys &rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk.k0[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk.k1[r],
                       (uint32_t)p0);
    }
    return c;
}

__device__ __forceinline__ uint32_t lane_of(uint4 w, int lane) {
    return lane == 0 ? w.x : lane == 1 ? w.y : lane == 2 ? w.z : w.w;
}

// ------------------------------------------------------------ division --
// Division of n < 2^31 by a fixed d >= 1 as a multiply-high, add and shift
// (the round-up multiplier of Granlund and Montgomery, "Division by invariant
// integers using multiplication", PLDI 1994): l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (mulhi(n, m) + n) >> l.
struct FastDiv {
    uint32_t d, m, l;
};

inline FastDiv make_fastdiv(uint32_t d) {
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    const uint64_t m = ((((uint64_t)1 << l) - d) << 32) / d + 1;
    return FastDiv{d, (uint32_t)m, l};
}

__device__ __forceinline__ FastDiv make_fastdiv_dev(uint32_t d) {
    const uint32_t l = d <= 1 ? 0u : 32u - __clz(d - 1);
    const uint64_t m = ((((uint64_t)1 << l) - d) << 32) / d + 1;
    return FastDiv{d, (uint32_t)m, l};
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv &f) {
    return (__umulhi(n, f.m) + n) >> f.l;
}

// ------------------------------------------------------------- geometry --
struct Geometry {
    int L;        // linear size (even)
    int Lh;       // L / 2 sites per row of one parity
    int P;        // row pitch in bytes (multiple of 4)
    int W;        // 32-bit words per row, P / 4
    int64_t half; // bytes of one parity half, L * L * P
};

// ------------------------------------------------- neighbour word assembly --
// O[0..NW-1]: words of the opposite-parity row that sits at the same (y, z),
// covering bytes [b0, b0 + 4 NW) of the row. Builds the +x and -x neighbour
// words of the own-parity sites in the same byte range. `o` is the own row's
// x offset ((p + y + z) & 1): for o = 0 site i sits at x = 2i, its +x
// neighbour is O[i] and its -x neighbour O[i-1]; for o = 1 (x = 2i + 1) they
// are O[i+1] and O[i]. `edge` is the byte just before the range (o = 0) or
// just after it (o = 1), `first` and `last` the row's bytes 0 and Lh - 1 for
// the periodic wrap. INSERT = false: the caller has already passed the row's
// first byte as `edge` when the range ends at the row's last site (rows
// without padding), so no wrap byte needs inserting.
template <int NW, bool INSERT = true>
__device__ __forceinline__ void x_neighbours(const uint32_t (&O)[NW], int o, int b0, int Lh,
                                             uint32_t edge, uint32_t first, uint32_t last,
                                             uint32_t (&xp)[NW], uint32_t (&xm)[NW]) {
    if (o == 0) {
        const uint32_t prev = (b0 == 0) ? last : edge;
#pragma unroll
        for (int j = 0; j < NW; ++j) {
            xp[j] = O[j];
            xm[j] = (O[j] << 8) | (j == 0 ? prev : (O[j - 1] >> 24));
        }
    } else {
#pragma unroll
        for (int j = 0; j < NW; ++j) {
            xm[j] = O[j];
            xp[j] = (O[j] >> 8) | ((j + 1 < NW ? (O[j + 1] & 0xFFu) : edge) << 24);
        }
        if constexpr (INSERT) {
            // the row's last site takes the row's first byte as its +x neighbour;
            // written branch-free per word so that xp stays in registers
            const int e = Lh - 1 - b0;  // position of the row's last site in this range
#pragma unroll
            for (int j = 0; j < NW; ++j) {
                const int pos = e - 4 * j;
                const bool here = pos >= 0 && pos < 4;
                const uint32_t sh = here ? 8u * (uint32_t)pos : 0u;
                const uint32_t m = here ? (0xFFu << sh) : 0u;
                xp[j] = (xp[j] & ~m) | ((first << sh) & m);
            }
        }
    }
}

// Mask of the byte lanes of word j (bytes b0 + 4j ..) that hold real sites.
__device__ __forceinline__ uint32_t valid_mask(int b0, int j, int Lh) {
    const int n = Lh - (b0 + 4 * j);
    if (n >= 4) return 0xFFFFFFFFu;
    if (n <= 0) return 0u;
    return 0xFFFFFFFFu >> (8 * (4 - n));
}

// 0xFF in every byte lane whose most significant bit is set, 0x00 elsewhere:
// prmt in its default mode with selector nibbles 8 + b takes byte b and
// replicates its sign over the lane (the __byte_perm intrinsic has no sign mode).
__device__ __forceinline__ uint32_t lanes_from_msb(uint32_t x) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %1, 0xBA98;" : "=r"(r) : "r"(x));
    return r;
}

// Bond word shifted so that the bit of direction k lands on bit 5 of each lane.
struct BondPlanes {
    uint32_t xp, yp, zp, xm, ym, zm;
};

__device__ __forceinline__ BondPlanes bond_planes(uint32_t B) {
    return {B << 5, B << 4, B << 3, B << 2, B << 1, B};
}

// 32 * (number of frustrated-or-not bonds whose J s_nb is negative) per lane:
// bit 5 of (neighbour ^ shifted bond) is set iff J s_nb = -1.
__device__ __forceinline__ uint32_t negative_terms(const BondPlanes &b, uint32_t xp, uint32_t xm,
                                                   uint32_t yp, uint32_t ym, uint32_t zp,
                                                   uint32_t zm) {
    constexpr uint32_t M = 0x20202020u;
    return ((xp ^ b.xp) & M) + ((xm ^ b.xm) & M) + ((yp ^ b.yp) & M) + ((ym ^ b.ym) & M) +
           ((zp ^ b.zp) & M) + ((zm ^ b.zm) & M);
}

// Per lane: 32 * u, u = number of unsatisfied bonds of the site (J s s_nb = -1),
// from the site's bond word B and its own spin word S. Bits 1..7 of a +-1 spin
// byte all hold its sign, so bits 0..5 of S >> 1 carry the own sign in every
// lane and bit k of B ^ (S >> 1) is the sign of J_k s; the shift that brings
// bit k to bit 5 and the XOR with the neighbour then give [J_k s s_nb = -1].
// (Bits 6, 7 of a lane never reach bit 5 of any lane under the left shifts.)
__device__ __forceinline__ uint32_t unsatisfied_count(uint32_t B, uint32_t S, uint32_t xp, uint32_t xm,
                                                      uint32_t yp, uint32_t ym, uint32_t zp, uint32_t zm) {
    return negative_terms(bond_planes(B ^ (S >> 1)), xp, xm, yp, ym, zp, zm);
}

// The elementary move on four lanes. With u unsatisfied bonds dH = 12 - 4u, so
// Eq. (flip-OK), 0 <= 4m - dH <= 12, reads 3 <= u + m <= 6 and Eq. (Creutz)
// gives m' = u + m - 3. Returns the byte mask of accepted lanes and updates
// D (daemons) in place.
__device__ __forceinline__ uint32_t creutz4(uint32_t u32, uint32_t &D, uint32_t valid) {
    const uint32_t t = (u32 >> 5) + D;         // u + m in 0..9 per lane
    const uint32_t v = t + 0x7D7D7D7Du;         // 0x80..0x83 <=> accepted
    const uint32_t am = lanes_from_msb(v & ~(v << 5)) & valid;  // bit 7 set and bit 2 clear
    D = (D & ~am) | (v & 0x03030303u & am);
    return am;
}

// Daemon value from a uniform word and the three refresh cut points:
// m = [u >= c0] + [u >= c1] + [u >= c2], taken as strict 32-bit compares
// [u > c - 1]. Valid for 1 <= c <= 2^32; every refresh cut point is
// >= floor(2^32 p(0)) >= 2^30, since p(0) = 1 / (1 + x + x^2 + x^3) >= 1/4.
__device__ __forceinline__ uint32_t daemon_from_uniform(uint32_t u, uint64_t c0, uint64_t c1,
                                                        uint64_t c2) {
    return (uint32_t)(u > (uint32_t)(c0 - 1)) + (uint32_t)(u > (uint32_t)(c1 - 1)) +
           (uint32_t)(u > (uint32_t)(c2 - 1));
}

}  // namespace micsa
