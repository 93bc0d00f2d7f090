/*
 * micsa_oracle.c -- plain CPU oracle for MicSA (test infrastructure only).
 *
 * Written from the paper's definitions: Eq. (Hamiltonian) for the energy,
 * Eq. (Creutz) and Eq. (flip-OK) for the elementary move, Eq.
 * (prob-daemons-walkers) for the daemon refresh, the procedure of Sec. 2.8 for
 * the order of operations. One site at a time, natural layout, int energies.
 * No blocking, no bit tricks, no shared code with the CUDA path.
 *
 * Planted mistakes: building with -DORC_MUTANT=k (k >= 1) compiles one
 * deliberate error into this file; the pin tests use those builds to show that
 * each pin fails when the arithmetic it guards is wrong.
 */
#include "micsa_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

enum { TAG_COUPLING = 0, TAG_SPIN = 1, TAG_DAEMON = 2, TAG_METRO = 3 };

/* ---------------------------------------------------------------- Philox -- */

/* Philox4x32 round constants from Salmon et al. (SC'11): the two multipliers
 * of the S-box and the two Weyl increments of the key schedule. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * x0;  /* 32x32 -> 64 bit products */
        uint64_t p1 = (uint64_t)PHILOX_M1 * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += PHILOX_W0;  /* key schedule: bump between rounds */
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void philox_seeded(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                          uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------- lattice -- */

static int64_t site_of(int L, int x, int y, int z) {
    return ((int64_t)z * L + y) * L + x;
}

static int wrap(int c, int L) {
    c %= L;
    return c < 0 ? c + L : c;
}

/* Counter word c0 and output lane of the Philox block used for the daemon
 * refresh and the Metropolis draws of site (x, y, z). */
static void quad_of(int L, int x, int y, int z, uint32_t *quad, int *lane) {
    int p = (x + y + z) & 1;
    int h = x >> 1;
    int64_t Q = (((int64_t)L + 1) / 2 + 3) / 4;
    *quad = (uint32_t)((((int64_t)p * L + z) * L + y) * Q + (h >> 2));
    *lane = h & 3;
}

/* Sum over the six neighbours y of J_xy s_y (the local field of Sec. 2.3).
 * Forward bonds of x are J[x][d]; the backward bond along d is the forward
 * bond of the neighbour x - e_d. */
static int local_field(int L, const int8_t *J, const int8_t *s, int x, int y, int z) {
    int64_t xp = site_of(L, wrap(x + 1, L), y, z), xm = site_of(L, wrap(x - 1, L), y, z);
    int64_t yp = site_of(L, x, wrap(y + 1, L), z), ym = site_of(L, x, wrap(y - 1, L), z);
    int64_t zp = site_of(L, x, y, wrap(z + 1, L)), zm = site_of(L, x, y, wrap(z - 1, L));
    int64_t c = site_of(L, x, y, z);
    int h = 0;
    h += J[c * 3 + 0] * s[xp];
    h += J[xm * 3 + 0] * s[xm];
    h += J[c * 3 + 1] * s[yp];
#if ORC_MUTANT == 3
    h += J[c * 3 + 1] * s[ym];  /* planted: -y neighbour read through the +y bond */
#else
    h += J[ym * 3 + 1] * s[ym];
#endif
    h += J[c * 3 + 2] * s[zp];
    h += J[zm * 3 + 2] * s[zm];
    return h;
}

int64_t orc_energy(int L, const int8_t *J, const int8_t *s) {
    int64_t H = 0;
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int64_t c = site_of(L, x, y, z);
                H -= J[c * 3 + 0] * s[c] * s[site_of(L, wrap(x + 1, L), y, z)];
                H -= J[c * 3 + 1] * s[c] * s[site_of(L, x, wrap(y + 1, L), z)];
                H -= J[c * 3 + 2] * s[c] * s[site_of(L, x, y, wrap(z + 1, L))];
            }
    return H;
}

int orc_delta_h(int L, const int8_t *J, const int8_t *s, int64_t site) {
    int x = (int)(site % L), y = (int)((site / L) % L), z = (int)(site / ((int64_t)L * L));
    return 2 * s[site] * local_field(L, J, s, x, y, z);
}

/* --------------------------------------------------------- initial data -- */

void orc_init_couplings(int L, uint64_t seed, int64_t sample, int8_t *J) {
    int64_t N = (int64_t)L * L * L;
    for (int64_t i = 0; i < N; ++i) {
        uint32_t w[4];
        philox_seeded(seed, (uint32_t)i, 0, (uint32_t)(sample << 2) | TAG_COUPLING, 0, w);
#if ORC_MUTANT == 5
        for (int d = 0; d < 3; ++d) J[i * 3 + d] = (w[0] >= 0x80000000u) ? -1 : 1;  /* planted: one word for all three bonds */
#else
        for (int d = 0; d < 3; ++d) J[i * 3 + d] = (w[d] >= 0x80000000u) ? -1 : 1;
#endif
    }
}

void orc_init_spins(int L, uint64_t seed, int64_t gid, int8_t *s) {
    int64_t N = (int64_t)L * L * L;
    for (int64_t i = 0; i < N; ++i) {
        uint32_t w[4];
        philox_seeded(seed, (uint32_t)i, 0, (uint32_t)(gid << 2) | TAG_SPIN, 0, w);
#if ORC_MUTANT == 6
        s[i] = (w[0] >= 0x40000000u) ? -1 : 1;  /* planted: p(s = -1) = 3/4 */
#else
        s[i] = (w[0] >= 0x80000000u) ? -1 : 1;
#endif
    }
}

/* ---------------------------------------------------------- thresholds -- */

static uint64_t cut_point(double c) {
    double v = floor(c * 4294967296.0);
    if (v >= 4294967296.0) return 4294967296ull;
    if (v <= 0.0) return 0;
    return (uint64_t)v;
}

/* Eq. (prob-daemons-walkers): p(n = 4m) = e^{-4 m beta} (1 - e^{-4 beta}) /
 * (1 - e^{-16 beta}), m = 0..3. With x = e^{-4 beta}: p(0) = (1 - x)/(1 - x^4),
 * p(m) = p(0) x^m. At x == 1 (beta -> 0) the four values tend to 1/4. */
int orc_daemon_thresholds(double T, uint64_t theta[3]) {
    if (!(T > 0.0) || isinf(T) || isnan(T)) return -1;
    double beta = 1.0 / T;
    double x = exp(-4.0 * beta);
    double p0;
    if (x == 1.0) {
        p0 = 0.25;
    } else {
        double x2 = x * x;
        double x4 = x2 * x2;
        p0 = (1.0 - x) / (1.0 - x4);
    }
    double p1 = p0 * x;
#if ORC_MUTANT == 4
    double p2 = p1 * x * x;  /* planted: wrong Boltzmann factor for m = 2 */
#else
    double p2 = p1 * x;
#endif
    double c0 = p0;
    double c1 = c0 + p1;
    double c2 = c1 + p2;
    theta[0] = cut_point(c0);
    theta[1] = cut_point(c1);
    theta[2] = cut_point(c2);
    return 0;
}

int orc_metro_thresholds(double T, uint64_t theta[3]) {
    if (!(T > 0.0) || isinf(T) || isnan(T)) return -1;
    double beta = 1.0 / T;
    for (int k = 0; k < 3; ++k) theta[k] = cut_point(exp(-beta * 4.0 * (k + 1)));
    return 0;
}

/* ------------------------------------------------------------- daemons -- */

int orc_refresh(int L, uint64_t seed, int64_t gid, int64_t t, double T, uint8_t *m) {
    uint64_t theta[3];
    if (orc_daemon_thresholds(T, theta)) return -1;
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                uint32_t quad, w[4];
                int lane;
                quad_of(L, x, y, z, &quad, &lane);
                philox_seeded(seed, quad, (uint32_t)t, (uint32_t)(gid << 2) | TAG_DAEMON,
                              (uint32_t)((uint64_t)t >> 32), w);
                uint64_t u = w[lane];
                int mm = (u >= theta[0]) + (u >= theta[1]) + (u >= theta[2]);
                m[site_of(L, x, y, z)] = (uint8_t)mm;
            }
    return 0;
}

/* The elementary move at one site: Eq. (Creutz) n -> n - dH, accepted iff the
 * result is legal, Eq. (flip-OK): 0 <= n - dH <= 12. */
static void creutz_move(int L, const int8_t *J, int8_t *s, uint8_t *m, int x, int y, int z) {
    int64_t c = site_of(L, x, y, z);
    int dH = 2 * s[c] * local_field(L, J, s, x, y, z);
    int n = 4 * m[c];
#if ORC_MUTANT == 2
    int n_new = n + dH;  /* planted: daemon absorbs the wrong sign */
#else
    int n_new = n - dH;
#endif
#if ORC_MUTANT == 1
    if (n_new >= 0 && n_new <= 16) {  /* planted: capacity one step too large */
        if (n_new > 12) n_new = 12;
#else
    if (n_new >= 0 && n_new <= 12) {
#endif
        s[c] = (int8_t)-s[c];
        m[c] = (uint8_t)(n_new / 4);
    }
}

void orc_half_sweep(int L, const int8_t *J, int8_t *s, uint8_t *m, int parity) {
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x)
                if (((x + y + z) & 1) == parity) creutz_move(L, J, s, m, x, y, z);
}

void orc_serial_sweep(int L, const int8_t *J, int8_t *s, uint8_t *m) {
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) creutz_move(L, J, s, m, x, y, z);
}

static int check_args(int L, int S, int R, int64_t n_sweeps, int serial) {
    if (L < 2 || S < 1 || R < 1 || n_sweeps < 0) return -1;
    if (!serial && (L & 1)) return -1;  /* checkerboard needs even L, Sec. 2.1 */
    return 0;
}

int orc_run(int L, int S, int R, uint64_t seed, const int8_t *J, int8_t *s, uint8_t *m,
            int64_t *t_io, const double *schedule, int64_t n_sweeps, int32_t interval,
            int serial) {
    if (check_args(L, S, R, n_sweeps, serial) || interval < 1) return -1;
    int64_t N = (int64_t)L * L * L;
    for (int64_t k = 0; k < n_sweeps; ++k) {
        int64_t t = *t_io + k;
        for (int a = 0; a < S; ++a) {
            const int8_t *Ja = J + (int64_t)a * N * 3;
            for (int r = 0; r < R; ++r) {
                int64_t gid = (int64_t)a * R + r;
                int8_t *sr = s + gid * N;
                uint8_t *mr = m + gid * N;
                if (t % interval == 0 && orc_refresh(L, seed, gid, t, schedule[k], mr)) return -1;
                if (serial) {
                    orc_serial_sweep(L, Ja, sr, mr);
                } else {
                    orc_half_sweep(L, Ja, sr, mr, 0);
                    orc_half_sweep(L, Ja, sr, mr, 1);
                }
            }
        }
    }
    *t_io += n_sweeps;
    return 0;
}

static int is_log_refresh_time(int64_t t) {
    /* t + 1 a power of two <=> t = 2^s - 1 */
    uint64_t v = (uint64_t)t + 1;
    return (v & (v - 1)) == 0;
}

int orc_run_logrefresh(int L, int S, int R, uint64_t seed, const int8_t *J, int8_t *s,
                       uint8_t *m, int64_t *t_io, const double *schedule, int64_t n_sweeps) {
    if (check_args(L, S, R, n_sweeps, 0)) return -1;
    int64_t N = (int64_t)L * L * L;
    for (int64_t k = 0; k < n_sweeps; ++k) {
        int64_t t = *t_io + k;
        for (int a = 0; a < S; ++a)
            for (int r = 0; r < R; ++r) {
                int64_t gid = (int64_t)a * R + r;
                if (is_log_refresh_time(t) &&
                    orc_refresh(L, seed, gid, t, schedule[k], m + gid * N))
                    return -1;
                orc_half_sweep(L, J + (int64_t)a * N * 3, s + gid * N, m + gid * N, 0);
                orc_half_sweep(L, J + (int64_t)a * N * 3, s + gid * N, m + gid * N, 1);
            }
    }
    *t_io += n_sweeps;
    return 0;
}

/* ------------------------------------------------- daemons and walkers -- */

static const int DIR_DX[6] = {1, 0, 0, -1, 0, 0};
static const int DIR_DY[6] = {0, 1, 0, 0, -1, 0};
static const int DIR_DZ[6] = {0, 0, 1, 0, 0, -1};

void orc_wander(int L, uint8_t *m, int dir, int parity) {
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                if (((x + y + z) & 1) != parity) continue;
                int64_t a = site_of(L, x, y, z);
                int64_t b = site_of(L, wrap(x + DIR_DX[dir], L), wrap(y + DIR_DY[dir], L),
                                    wrap(z + DIR_DZ[dir], L));
                uint8_t tmp = m[a];
                m[a] = m[b];
                m[b] = tmp;
            }
}

int orc_run_ex(int L, int S, int R, int gamma, int walkers, uint64_t seed, const int8_t *J, int8_t *s,
               uint8_t *m, int64_t *t_io, const double *schedule, int64_t n_steps, int32_t interval) {
    if (check_args(L, S, R, n_steps, 0) || gamma < 1 || interval < 0) return -1;
    int64_t N = (int64_t)L * L * L;
    for (int64_t k = 0; k < n_steps; ++k) {
        int64_t t = *t_io + k;
        int refresh = interval > 0 ? (t % interval == 0) : is_log_refresh_time(t);
        for (int a = 0; a < S; ++a)
            for (int r = 0; r < R; ++r) {
                int64_t gid = (int64_t)a * R + r;
                const int8_t *Ja = J + (int64_t)a * N * 3;
                int8_t *sr = s + gid * N;
                uint8_t *mr = m + gid * gamma * N;  /* daemon alpha at mr + alpha * N */
                if (refresh)
                    for (int al = 0; al < gamma; ++al)
                        if (orc_refresh(L, seed, gid * gamma + al, t, schedule[k], mr + al * N)) return -1;
                for (int al = 0; al < gamma; ++al) {
                    orc_half_sweep(L, Ja, sr, mr + al * N, 0);
                    orc_half_sweep(L, Ja, sr, mr + al * N, 1);
                }
                if (walkers)
                    for (int al = 0; al < gamma; ++al) orc_wander(L, mr + al * N, al % 6, (int)(t & 1));
            }
    }
    *t_io += n_steps;
    return 0;
}

/* ---------------------------------------------------------- Metropolis -- */

static void metro_move(int L, uint64_t seed, int64_t gid, int64_t t, const uint64_t theta[3],
                       const int8_t *J, int8_t *s, int x, int y, int z) {
    int64_t c = site_of(L, x, y, z);
    int dH = 2 * s[c] * local_field(L, J, s, x, y, z);
    int accept;
    if (dH <= 0) {
        accept = 1;
    } else {
        uint32_t quad, w[4];
        int lane;
        quad_of(L, x, y, z, &quad, &lane);
        philox_seeded(seed, quad, (uint32_t)t, (uint32_t)(gid << 2) | TAG_METRO,
                      (uint32_t)((uint64_t)t >> 32), w);
        accept = (uint64_t)w[lane] < theta[dH / 4 - 1];
    }
    if (accept) s[c] = (int8_t)-s[c];
}

int orc_run_metropolis(int L, int S, int R, uint64_t seed, const int8_t *J, int8_t *s,
                       int64_t *t_io, const double *schedule, int64_t n_sweeps, int serial) {
    if (check_args(L, S, R, n_sweeps, serial)) return -1;
    int64_t N = (int64_t)L * L * L;
    for (int64_t k = 0; k < n_sweeps; ++k) {
        int64_t t = *t_io + k;
        uint64_t theta[3];
        if (orc_metro_thresholds(schedule[k], theta)) return -1;
        for (int a = 0; a < S; ++a)
            for (int r = 0; r < R; ++r) {
                int64_t gid = (int64_t)a * R + r;
                const int8_t *Ja = J + (int64_t)a * N * 3;
                int8_t *sr = s + gid * N;
                for (int pass = 0; pass < (serial ? 1 : 2); ++pass)
                    for (int z = 0; z < L; ++z)
                        for (int y = 0; y < L; ++y)
                            for (int x = 0; x < L; ++x)
                                if (serial || ((x + y + z) & 1) == pass)
                                    metro_move(L, seed, gid, t, theta, Ja, sr, x, y, z);
            }
    }
    *t_io += n_sweeps;
    return 0;
}

/* --------------------------------------------------------- observables -- */

void orc_measure(int L, int S, int R, const int8_t *J, const int8_t *s, const uint8_t *m,
                 int64_t *energy, int64_t *aux, int64_t *overlap) {
    int64_t N = (int64_t)L * L * L;
    int64_t pair = 0;
    for (int a = 0; a < S; ++a) {
        for (int r = 0; r < R; ++r) {
            int64_t gid = (int64_t)a * R + r;
            if (energy) energy[gid] = orc_energy(L, J + (int64_t)a * N * 3, s + gid * N);
            if (aux) {
                int64_t sum = 0;
                for (int64_t i = 0; i < N; ++i) sum += 4 * m[gid * N + i];
                aux[gid] = sum;
            }
        }
        for (int ra = 0; ra < R; ++ra)
            for (int rb = ra + 1; rb < R; ++rb, ++pair) {
                if (!overlap) continue;
                const int8_t *sa = s + ((int64_t)a * R + ra) * N;
                const int8_t *sb = s + ((int64_t)a * R + rb) * N;
                int64_t q = 0;
#if ORC_MUTANT == 7
                for (int64_t i = 0; i < N; ++i) q += sa[i] * sa[i];  /* planted: replica a with itself */
#else
                for (int64_t i = 0; i < N; ++i) q += sa[i] * sb[i];
#endif
                overlap[pair] = q;
            }
    }
}

/* --------------------------------------------------------- correlation -- */

int orc_correlation(int L, int S, int R, const int8_t *s, int64_t *G) {
    if (R < 2) return -1;
    int64_t N = (int64_t)L * L * L;
    for (int a = 0; a < S; ++a) {
        int64_t *Ga = G + (int64_t)a * L;
        for (int r = 0; r < L; ++r) Ga[r] = 0;
        for (int ra = 0; ra < R; ++ra)
            for (int rb = ra + 1; rb < R; ++rb) {
                const int8_t *sa = s + ((int64_t)a * R + ra) * N;
                const int8_t *sb = s + ((int64_t)a * R + rb) * N;
                for (int z = 0; z < L; ++z)
                    for (int y = 0; y < L; ++y)
                        for (int x = 0; x < L; ++x) {
                            int64_t c = site_of(L, x, y, z);
                            int qx = sa[c] * sb[c];
                            for (int r = 0; r < L; ++r) {
                                int64_t ex = site_of(L, wrap(x + r, L), y, z);
                                int64_t ey = site_of(L, x, wrap(y + r, L), z);
                                int64_t ez = site_of(L, x, y, wrap(z + r, L));
                                Ga[r] += qx * (sa[ex] * sb[ex] + sa[ey] * sb[ey] + sa[ez] * sb[ez]);
                            }
                        }
            }
    }
    return 0;
}

/* --------------------------------------------------------- enumeration -- */

int orc_enumerate_dos(int L, const int8_t *J, int64_t *counts) {
    int64_t N = (int64_t)L * L * L;
    if (N > 30) return -1;
    int8_t *s = (int8_t *)malloc((size_t)N);
    if (!s) return -1;
    for (int64_t i = 0; i < N; ++i) s[i] = 1;
    int64_t E = orc_energy(L, J, s);
    memset(counts, 0, sizeof(int64_t) * (size_t)(6 * N + 1));
    counts[E + 3 * N] += 1;
    /* reflected Gray code: step i flips the spin at the lowest set bit of i */
    uint64_t total = 1ull << N;
    for (uint64_t i = 1; i < total; ++i) {
        int64_t k = __builtin_ctzll(i);
        E += orc_delta_h(L, J, s, k);
        s[k] = (int8_t)-s[k];
        counts[E + 3 * N] += 1;
    }
    free(s);
    return 0;
}

int orc_all_energies(int L, const int8_t *J, int64_t *E) {
    int64_t N = (int64_t)L * L * L;
    if (N > 24) return -1;
    int8_t *s = (int8_t *)malloc((size_t)N);
    if (!s) return -1;
    for (uint64_t st = 0; st < (1ull << N); ++st) {
        for (int64_t i = 0; i < N; ++i) s[i] = ((st >> i) & 1) ? -1 : 1;
        E[st] = orc_energy(L, J, s);
    }
    free(s);
    return 0;
}

static void spins_from_index(int N, uint32_t st, int8_t *s) {
    for (int i = 0; i < N; ++i) s[i] = ((st >> i) & 1) ? -1 : 1;
}

static uint32_t index_from_spins(int N, const int8_t *s) {
    uint32_t st = 0;
    for (int i = 0; i < N; ++i)
        if (s[i] < 0) st |= 1u << i;
    return st;
}

int orc_l2_transition_micsa(const int8_t *J, const double pm[4], double *P) {
    const int L = 2, N = 8;
    memset(P, 0, sizeof(double) * 256 * 256);
    int8_t s[8];
    uint8_t m[8];
    for (uint32_t a = 0; a < 256; ++a) {
        for (uint32_t d = 0; d < (1u << (2 * N)); ++d) {
            double w = 1.0;
            for (int i = 0; i < N; ++i) {
                m[i] = (uint8_t)((d >> (2 * i)) & 3);
                w *= pm[m[i]];
            }
            spins_from_index(N, a, s);
            orc_half_sweep(L, J, s, m, 0);
            orc_half_sweep(L, J, s, m, 1);
            P[a * 256 + index_from_spins(N, s)] += w;
        }
    }
    return 0;
}

/* Half-sweep transition matrix of Metropolis: the sites of one parity flip
 * independently given the other parity (Sec. 2.1 separability), each with
 * probability 1 (dH <= 0) or theta/2^32. */
static void metro_half_matrix(const int8_t *J, const uint64_t theta[3], int parity, double *Ph) {
    const int L = 2, N = 8;
    int sites[4], ns = 0;
    for (int i = 0; i < N; ++i) {
        int x = i % 2, y = (i / 2) % 2, z = i / 4;
        if (((x + y + z) & 1) == parity) sites[ns++] = i;
    }
    memset(Ph, 0, sizeof(double) * 256 * 256);
    int8_t s[8];
    for (uint32_t a = 0; a < 256; ++a) {
        double pflip[4];
        spins_from_index(N, a, s);
        for (int k = 0; k < ns; ++k) {
            int dH = orc_delta_h(L, J, s, sites[k]);
            pflip[k] = dH <= 0 ? 1.0 : (double)theta[dH / 4 - 1] / 4294967296.0;
        }
        for (uint32_t sub = 0; sub < (1u << ns); ++sub) {
            double w = 1.0;
            uint32_t b = a;
            for (int k = 0; k < ns; ++k) {
                if ((sub >> k) & 1) {
                    w *= pflip[k];
                    b ^= 1u << sites[k];
                } else {
                    w *= 1.0 - pflip[k];
                }
            }
            Ph[a * 256 + b] += w;
        }
    }
}

int orc_l2_transition_metro(const int8_t *J, double T, double *P) {
    uint64_t theta[3];
    if (orc_metro_thresholds(T, theta)) return -1;
    double *Pe = (double *)malloc(sizeof(double) * 256 * 256);
    double *Po = (double *)malloc(sizeof(double) * 256 * 256);
    if (!Pe || !Po) {
        free(Pe);
        free(Po);
        return -1;
    }
    metro_half_matrix(J, theta, 0, Pe);
    metro_half_matrix(J, theta, 1, Po);
    for (int a = 0; a < 256; ++a)
        for (int b = 0; b < 256; ++b) {
            double acc = 0.0;
            for (int c = 0; c < 256; ++c) acc += Pe[a * 256 + c] * Po[c * 256 + b];
            P[a * 256 + b] = acc;
        }
    free(Pe);
    free(Po);
    return 0;
}
