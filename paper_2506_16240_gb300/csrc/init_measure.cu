// init_measure.cu -- coupling and spin initialisation from the seed, layout
// conversion between the caller's natural order and the sublattice-split
// device layout, and the exact integer observables of Sec. 3 / App. C.
#include <algorithm>

#include "micsa_internal.h"

namespace micsa {

Geometry make_geometry(int L) {
    Geometry g;
    g.L = L;
    g.Lh = L / 2;
    g.W = (g.Lh + 3) / 4;
    g.P = 4 * g.W;
    g.half = (int64_t)L * L * g.P;
    return g;
}

// byte offset of natural site (x, y, z) inside its parity half
__device__ __forceinline__ int64_t split_offset(const Geometry &g, int x, int y, int z,
                                                int *parity) {
    *parity = (x + y + z) & 1;
    return ((int64_t)z * g.L + y) * g.P + (x >> 1);
}

__device__ __forceinline__ void site_xyz(const Geometry &g, int64_t site, int &x, int &y, int &z) {
    x = (int)(site % g.L);
    y = (int)((site / g.L) % g.L);
    z = (int)(site / ((int64_t)g.L * g.L));
}

__device__ __forceinline__ uint32_t wrapm(int c, int L) { return (uint32_t)(c < 0 ? c + L : c >= L ? c - L : c); }

// ------------------------------------------------------------ couplings --
// Forward bonds of a site from the seed: J_{+d} = -1 iff word d >= 2^31.
__device__ __forceinline__ uint32_t forward_bits(uint32_t site, int sample, uint32_t k0, uint32_t k1) {
    const uint4 w = philox4x32_10(make_uint4(site, 0u, ((uint32_t)sample << 2) | kTagCoupling, 0u), k0, k1);
    return (w.x >> 31) | ((w.y >> 31) << 1) | ((w.z >> 31) << 2);
}

__global__ void init_couplings_kernel(uint8_t *bonds, Geometry g, int S, uint32_t k0, uint32_t k1) {
    const int64_t N = (int64_t)g.L * g.L * g.L;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= N * S) return;
    const int sample = (int)(tid / N);
    const int64_t site = tid - (int64_t)sample * N;
    int x, y, z;
    site_xyz(g, site, x, y, z);
    const uint32_t fwd = forward_bits((uint32_t)site, sample, k0, k1);
    const int64_t sxm = ((int64_t)z * g.L + y) * g.L + wrapm(x - 1, g.L);
    const int64_t sym = ((int64_t)z * g.L + wrapm(y - 1, g.L)) * g.L + x;
    const int64_t szm = ((int64_t)wrapm(z - 1, g.L) * g.L + y) * g.L + x;
    const uint32_t bxm = forward_bits((uint32_t)sxm, sample, k0, k1) & 1u;
    const uint32_t bym = (forward_bits((uint32_t)sym, sample, k0, k1) >> 1) & 1u;
    const uint32_t bzm = (forward_bits((uint32_t)szm, sample, k0, k1) >> 2) & 1u;
    int p;
    const int64_t off = split_offset(g, x, y, z, &p);
    bonds[(int64_t)(sample * 2 + p) * g.half + off] = (uint8_t)(fwd | (bxm << 3) | (bym << 4) | (bzm << 5));
}

// J_nat[S][N][3] of +-1 -> bond bytes
__global__ void pack_couplings_kernel(uint8_t *bonds, const int8_t *J, Geometry g, int S) {
    const int64_t N = (int64_t)g.L * g.L * g.L;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= N * S) return;
    const int sample = (int)(tid / N);
    const int64_t site = tid - (int64_t)sample * N;
    int x, y, z;
    site_xyz(g, site, x, y, z);
    const int8_t *Js = J + (int64_t)sample * N * 3;
    const int64_t sxm = ((int64_t)z * g.L + y) * g.L + wrapm(x - 1, g.L);
    const int64_t sym = ((int64_t)z * g.L + wrapm(y - 1, g.L)) * g.L + x;
    const int64_t szm = ((int64_t)wrapm(z - 1, g.L) * g.L + y) * g.L + x;
    uint32_t b = 0;
    b |= (uint32_t)(Js[site * 3 + 0] < 0) << 0;
    b |= (uint32_t)(Js[site * 3 + 1] < 0) << 1;
    b |= (uint32_t)(Js[site * 3 + 2] < 0) << 2;
    b |= (uint32_t)(Js[sxm * 3 + 0] < 0) << 3;
    b |= (uint32_t)(Js[sym * 3 + 1] < 0) << 4;
    b |= (uint32_t)(Js[szm * 3 + 2] < 0) << 5;
    int p;
    const int64_t off = split_offset(g, x, y, z, &p);
    bonds[(int64_t)(sample * 2 + p) * g.half + off] = (uint8_t)b;
}

__global__ void unpack_couplings_kernel(int8_t *J, const uint8_t *bonds, Geometry g, int S) {
    const int64_t N = (int64_t)g.L * g.L * g.L;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= N * S) return;
    const int sample = (int)(tid / N);
    const int64_t site = tid - (int64_t)sample * N;
    int x, y, z;
    site_xyz(g, site, x, y, z);
    int p;
    const int64_t off = split_offset(g, x, y, z, &p);
    const uint32_t b = bonds[(int64_t)(sample * 2 + p) * g.half + off];
    int8_t *Js = J + (int64_t)sample * N * 3 + site * 3;
    Js[0] = (b & 1u) ? -1 : 1;
    Js[1] = (b & 2u) ? -1 : 1;
    Js[2] = (b & 4u) ? -1 : 1;
}

// ---------------------------------------------------------------- spins --
__global__ void init_spins_kernel(int8_t *spins, Geometry g, int64_t n_gid, uint32_t k0, uint32_t k1) {
    const int64_t N = (int64_t)g.L * g.L * g.L;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= N * n_gid) return;
    const int64_t gid = tid / N;
    const int64_t site = tid - gid * N;
    int x, y, z;
    site_xyz(g, site, x, y, z);
    const uint4 w = philox4x32_10(make_uint4((uint32_t)site, 0u, ((uint32_t)gid << 2) | kTagSpin, 0u), k0, k1);
    int p;
    const int64_t off = split_offset(g, x, y, z, &p);
    spins[(gid * 2 + p) * g.half + off] = (w.x >> 31) ? (int8_t)-1 : (int8_t)1;
}

__global__ void convert_sites_kernel(uint8_t *split, uint8_t *natural, Geometry g, int64_t n,
                                     bool to_split) {
    const int64_t N = (int64_t)g.L * g.L * g.L;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= N * n) return;
    const int64_t k = tid / N;
    const int64_t site = tid - k * N;
    int x, y, z;
    site_xyz(g, site, x, y, z);
    int p;
    const int64_t off = (k * 2) * g.half + split_offset(g, x, y, z, &p);
    if (to_split)
        split[off + p * g.half] = natural[tid];
    else
        natural[tid] = split[off + p * g.half];
}

static inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t launch_init_couplings(uint8_t *bonds, Geometry g, int S, uint32_t k0, uint32_t k1,
                                  cudaStream_t st) {
    const int64_t n = (int64_t)g.L * g.L * g.L * S;
    init_couplings_kernel<<<blocks_for(n, 256), 256, 0, st>>>(bonds, g, S, k0, k1);
    return cudaGetLastError();
}

cudaError_t launch_init_spins(int8_t *spins, Geometry g, int S, int R, uint32_t k0, uint32_t k1,
                              cudaStream_t st) {
    const int64_t n = (int64_t)g.L * g.L * g.L * S * R;
    init_spins_kernel<<<blocks_for(n, 256), 256, 0, st>>>(spins, g, (int64_t)S * R, k0, k1);
    return cudaGetLastError();
}

cudaError_t launch_pack_couplings(uint8_t *bonds, const int8_t *J_nat, Geometry g, int S,
                                  cudaStream_t st) {
    const int64_t n = (int64_t)g.L * g.L * g.L * S;
    pack_couplings_kernel<<<blocks_for(n, 256), 256, 0, st>>>(bonds, J_nat, g, S);
    return cudaGetLastError();
}

cudaError_t launch_unpack_couplings(int8_t *J_nat, const uint8_t *bonds, Geometry g, int S,
                                    cudaStream_t st) {
    const int64_t n = (int64_t)g.L * g.L * g.L * S;
    unpack_couplings_kernel<<<blocks_for(n, 256), 256, 0, st>>>(J_nat, bonds, g, S);
    return cudaGetLastError();
}

// Index of the first byte of v[0, n) that is not a spin or coupling (+-1,
// mode 0) or not a daemon value (0..3, mode 1), min-reduced into *first, which
// the launcher presets to all ones (no such byte).
__global__ void first_invalid_kernel(const uint8_t *v, int64_t n, int mode, unsigned long long *first) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = v[i];
        if (mode == 0 ? (b != 0x01u && b != 0xFFu) : (b > 3u)) atomicMin(first, (unsigned long long)i);
    }
}

cudaError_t launch_first_invalid(const uint8_t *v, int64_t n, int mode, unsigned long long *first,
                                 cudaStream_t st) {
    if (cudaError_t e = cudaMemsetAsync(first, 0xFF, sizeof(unsigned long long), st)) return e;
    const unsigned blocks = n <= 0 ? 1u : std::min(blocks_for(n, 256), 4096u);  // grid-stride beyond
    first_invalid_kernel<<<blocks, 256, 0, st>>>(v, n, mode, first);
    return cudaGetLastError();
}

cudaError_t launch_convert_sites(uint8_t *split, uint8_t *natural, Geometry g, int64_t n,
                                 bool to_split, cudaStream_t st) {
    const int64_t total = (int64_t)g.L * g.L * g.L * n;
    convert_sites_kernel<<<blocks_for(total, 256), 256, 0, st>>>(split, natural, g, n, to_split);
    return cudaGetLastError();
}

// ---------------------------------------------------------- observables --
// One thread per (row, word) of one sample (blockIdx.y = sample). Per word:
//   energy (even sites only, each bond has exactly one even end for even L):
//     H = sum_even (2u - 6), u = unsatisfied bonds of the site;
//   H_aux = 4 * sum of m over both parities;
//   overlap of pair (a, b) = sum over sites of s_a s_b = n_valid - 2 n_differ.
// Per-block sums go through shared memory, then one atomic per block and
// quantity into out = [energy S*R | aux S*R | overlap S*R(R-1)/2].
__global__ void __launch_bounds__(256) measure_kernel(const int8_t *spins, const uint8_t *daemons,
                                                      const uint8_t *bonds, Geometry g, int S, int R,
                                                      int gamma, unsigned long long *out) {
    extern __shared__ long long acc[];  // [2R + R(R-1)/2]
    const int npair = R * (R - 1) / 2;
    const int nq = 2 * R + npair;
    for (int i = threadIdx.x; i < nq; i += blockDim.x) acc[i] = 0;
    __syncthreads();

    const int sample = blockIdx.y;
    const int64_t words = (int64_t)g.L * g.L * g.W;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = tid < words;
    const int row = active ? (int)(tid / g.W) : 0;
    const int wj = active ? (int)(tid - (int64_t)row * g.W) : 0;
    const int y = row % g.L, z = row / g.L;
    const int b0 = wj * 4;
    const uint32_t valid = active ? valid_mask(b0, 0, g.Lh) : 0u;
    const int nvalid = __popc(valid) / 8;
    const int lane = threadIdx.x & 31;

    // geometry of the even-site energy (p = 0)
    const int o = (y + z) & 1;
    const int yp = (y + 1 == g.L) ? 0 : y + 1, ym = (y == 0) ? g.L - 1 : y - 1;
    const int zp = (z + 1 == g.L) ? 0 : z + 1, zm = (z == 0) ? g.L - 1 : z - 1;
    const int64_t off_c = (int64_t)row * g.P + b0;
    const int64_t row0 = (int64_t)row * g.P;
    uint32_t Bw = 0;
    if (active) Bw = *reinterpret_cast<const uint32_t *>(bonds + (int64_t)(sample * 2) * g.half + off_c);

    for (int r = 0; r < R; ++r) {
        const int64_t gid = (int64_t)sample * R + r;
        int e_part = 0, a_part = 0;
        if (active) {
            const int8_t *even = spins + (gid * 2) * g.half;
            const int8_t *odd = even + g.half;
            const uint32_t S0 = *reinterpret_cast<const uint32_t *>(even + off_c);
            uint32_t O[1] = {*reinterpret_cast<const uint32_t *>(odd + off_c)};
            const uint32_t Oyp = *reinterpret_cast<const uint32_t *>(odd + ((int64_t)z * g.L + yp) * g.P + b0);
            const uint32_t Oym = *reinterpret_cast<const uint32_t *>(odd + ((int64_t)z * g.L + ym) * g.P + b0);
            const uint32_t Ozp = *reinterpret_cast<const uint32_t *>(odd + ((int64_t)zp * g.L + y) * g.P + b0);
            const uint32_t Ozm = *reinterpret_cast<const uint32_t *>(odd + ((int64_t)zm * g.L + y) * g.P + b0);
            uint32_t edge = 0, first = 0, last = 0;
            if (o == 0) {
                if (b0 == 0) last = (uint8_t)odd[row0 + g.Lh - 1];
                else edge = (uint8_t)odd[off_c - 1];
            } else {
                if (b0 + 4 <= g.Lh - 1) edge = (uint8_t)odd[off_c + 4];
                else first = (b0 == 0) ? (O[0] & 0xFFu) : (uint8_t)odd[row0];
            }
            uint32_t xp[1], xm[1];
            x_neighbours<1>(O, o, b0, g.Lh, edge, first, last, xp, xm);
            const uint32_t u32 = unsatisfied_count(Bw, S0, xp[0], xm[0], Oyp, Oym, Ozp, Ozm) & valid;
            const uint32_t usum = ((u32 >> 5) * 0x01010101u) >> 24;  // sum of the four lanes
            e_part = 2 * (int)usum - 6 * nvalid;
            for (int al = 0; al < gamma; ++al) {  // every daemon family (Sec. 2.2: H_aux sums them all)
                const int64_t fam = gid * gamma + al;
                const uint32_t D0 = *reinterpret_cast<const uint32_t *>(daemons + (fam * 2) * g.half + off_c);
                const uint32_t D1 = *reinterpret_cast<const uint32_t *>(daemons + (fam * 2 + 1) * g.half + off_c);
                a_part += 4 * (int)((((D0 & valid) * 0x01010101u) >> 24) + (((D1 & valid) * 0x01010101u) >> 24));
            }
        }
        e_part = __reduce_add_sync(0xFFFFFFFFu, e_part);
        a_part = __reduce_add_sync(0xFFFFFFFFu, a_part);
        if (lane == 0) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&acc[r]), (unsigned long long)(long long)e_part);
            atomicAdd(reinterpret_cast<unsigned long long *>(&acc[R + r]), (unsigned long long)(long long)a_part);
        }
    }
    int pair = 0;
    for (int ra = 0; ra < R; ++ra)
        for (int rb = ra + 1; rb < R; ++rb, ++pair) {
            int q_part = 0;
            if (active) {
                for (int par = 0; par < 2; ++par) {
                    const int64_t base_a = (((int64_t)sample * R + ra) * 2 + par) * g.half + off_c;
                    const int64_t base_b = (((int64_t)sample * R + rb) * 2 + par) * g.half + off_c;
                    const uint32_t Sa = *reinterpret_cast<const uint32_t *>(spins + base_a);
                    const uint32_t Sb = *reinterpret_cast<const uint32_t *>(spins + base_b);
                    const int ndiff = __popc((Sa ^ Sb) & 0x20202020u & valid);
                    q_part += nvalid - 2 * ndiff;
                }
            }
            q_part = __reduce_add_sync(0xFFFFFFFFu, q_part);
            if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long *>(&acc[2 * R + pair]), (unsigned long long)(long long)q_part);
        }
    __syncthreads();
    for (int i = threadIdx.x; i < nq; i += blockDim.x) {
        long long v = acc[i];
        if (v == 0) continue;
        int64_t dst;
        if (i < R) dst = (int64_t)sample * R + i;
        else if (i < 2 * R) dst = (int64_t)S * R + (int64_t)sample * R + (i - R);
        else dst = 2 * (int64_t)S * R + (int64_t)sample * npair + (i - 2 * R);
        atomicAdd(out + dst, (unsigned long long)v);
    }
}

// ------------------------------------------------- four-point correlation --
// q_x = s^a_x s^b_x of every replica pair a < b of every sample, natural layout:
// q[(sample * npair + pair) * N + site].
__global__ void overlap_field_kernel(int8_t *q, const int8_t *spins, Geometry g, int S, int R) {
    const int64_t N = (int64_t)g.L * g.L * g.L;
    const int npair = R * (R - 1) / 2;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= N * S * npair) return;
    const int64_t item = tid / N;
    const int64_t site = tid - item * N;
    const int sample = (int)(item / npair);
    int pair = (int)(item - (int64_t)sample * npair), ra = 0;
    while (pair >= R - 1 - ra) {  // pair index -> (ra, rb), lexicographic
        pair -= R - 1 - ra;
        ++ra;
    }
    const int rb = ra + 1 + pair;
    int x, y, z;
    site_xyz(g, site, x, y, z);
    int p;
    const int64_t in_half = split_offset(g, x, y, z, &p);
    const int64_t off = in_half + (int64_t)p * g.half;
    const int8_t sa = spins[(((int64_t)sample * R + ra) * 2) * g.half + off];
    const int8_t sb = spins[(((int64_t)sample * R + rb) * 2) * g.half + off];
    q[tid] = (int8_t)(sa * sb);
}

// G[sample][r] += sum over the block's lines along axis d of sum_i q_i q_{i+r}.
// Block: x = r (L threads), y = lines; grid: (line groups, axis, sample * pair).
__global__ void correlation_kernel(const int8_t *q, int L, int npair, unsigned long long *G) {
    extern __shared__ long long gsum[];  // [L]
    const int r = threadIdx.x;
    for (int i = threadIdx.y * blockDim.x + threadIdx.x; i < L; i += blockDim.x * blockDim.y) gsum[i] = 0;
    __syncthreads();
    const int64_t N = (int64_t)L * L * L;
    const int axis = blockIdx.y;
    const int item = blockIdx.z;  // sample * npair + pair
    const int64_t line = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
    if (line < (int64_t)L * L) {
        // the line's first site and stride along the axis
        const int u = (int)(line % L), v = (int)(line / L);
        int64_t base, stride;
        if (axis == 0) { base = ((int64_t)v * L + u) * L; stride = 1; }
        else if (axis == 1) { base = (int64_t)v * L * L + u; stride = L; }
        else { base = (int64_t)v * L + u; stride = (int64_t)L * L; }
        const int8_t *ql = q + (int64_t)item * N + base;
        int acc = 0;
        int j = r;
        for (int i = 0; i < L; ++i) {
            acc += ql[i * stride] * ql[j * stride];
            j = (j + 1 == L) ? 0 : j + 1;
        }
        atomicAdd(reinterpret_cast<unsigned long long *>(&gsum[r]), (unsigned long long)(long long)acc);
    }
    __syncthreads();
    const int sample = item / npair;
    for (int i = threadIdx.y * blockDim.x + threadIdx.x; i < L; i += blockDim.x * blockDim.y)
        if (gsum[i]) atomicAdd(G + (int64_t)sample * L + i, (unsigned long long)gsum[i]);
}

cudaError_t launch_correlation(const int8_t *spins, Geometry g, int S, int R, int8_t *q_scratch,
                               unsigned long long *G, cudaStream_t st) {
    const int64_t N = (int64_t)g.L * g.L * g.L;
    const int npair = R * (R - 1) / 2;
    const int64_t total = N * S * npair;
    overlap_field_kernel<<<blocks_for(total, 256), 256, 0, st>>>(q_scratch, spins, g, S, R);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int ly = g.L >= 1024 ? 1 : 1024 / g.L;
    const dim3 block((unsigned)g.L, (unsigned)ly);
    const dim3 grid((unsigned)(((int64_t)g.L * g.L + ly - 1) / ly), 3, (unsigned)(S * npair));
    correlation_kernel<<<grid, block, sizeof(long long) * g.L, st>>>(q_scratch, g.L, npair, G);
    return cudaGetLastError();
}

cudaError_t launch_measure(const int8_t *spins, const uint8_t *daemons, const uint8_t *bonds,
                           Geometry g, int S, int R, int gamma, unsigned long long *out, cudaStream_t st) {
    const int64_t words = (int64_t)g.L * g.L * g.W;
    const int nq = 2 * R + R * (R - 1) / 2;
    dim3 grid(blocks_for(words, 256), (unsigned)S);
    const size_t smem = sizeof(long long) * nq;  // 67 KB at R = 128
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(measure_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    measure_kernel<<<grid, 256, smem, st>>>(spins, daemons, bonds, g, S, R, gamma, out);
    return cudaGetLastError();
}

}  // namespace micsa
