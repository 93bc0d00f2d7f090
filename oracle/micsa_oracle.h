/*
 * micsa_oracle.h -- plain, slow, single-threaded CPU oracle for microcanonical
 * simulated annealing (MicSA) on the 3D Edwards-Anderson +-J spin glass.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call
 * this code: only the tests, the smoke check and the CPU baseline of the
 * benchmark do. It shares no source with the CUDA library.
 *
 * Layout: natural order, site = (z*L + y)*L + x, x fastest. Couplings are
 * stored as the three forward bonds of each site, J[site*3 + d] = +-1 for the
 * bond to site + e_d, d = 0 (x), 1 (y), 2 (z), periodic boundaries (Sec. 2.1,
 * Eq. Hamiltonian). Spins are int8 +-1. A daemon is stored as m in {0,1,2,3};
 * its energy is n = 4m (Sec. 2.4 and Sec. 2.5).
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), keyed by the 64-bit seed. The paper
 * names no generator; the counter layout below is this project's reading:
 *   key      = (seed & 0xffffffff, seed >> 32)
 *   coupling : ctr = (site, 0, (sample << 2) | 0, 0); word d >= 2^31  <=> J_{+d} = -1
 *   spin     : ctr = (site, 0, (gid << 2) | 1, 0);    word 0 >= 2^31  <=> s = -1
 *   daemon   : ctr = (quad, t mod 2^32, (gid << 2) | 2, t >> 32); u = word[lane]
 *   metropolis: ctr = (quad, t mod 2^32, (gid << 2) | 3, t >> 32); u = word[lane]
 * with gid = sample * R + replica, t the global sweep index, h = x >> 1,
 * Q = (ceil(L/2) + 3) / 4, quad = ((p*L + z)*L + y)*Q + (h >> 2), lane = h & 3 and
 * p = (x + y + z) & 1 the site parity. Four same-parity sites along x share
 * one Philox block.
 *
 * Parity status of each function is stated beside it; every function here is
 * pinned by a -m "not gpu" test (tests/test_oracle_*.py).
 */
#ifndef MICSA_ORACLE_H
#define MICSA_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32-10 block function (Salmon et al. SC'11, Sec. 3, the Philox
 * S-box with the published multipliers and Weyl key schedule).
 * Pinned against cuRAND's host Philox4_32_10 generator. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Refresh cut points for a daemon at temperature T, Eq. (prob-daemons-walkers):
 * theta[k] = min(floor(c_k * 2^32), 2^32), c_k = p(0) + ... + p(k);
 * m = [u >= theta0] + [u >= theta1] + [u >= theta2]. Returns 0, or -1 if T is
 * not a finite positive number. */
int orc_daemon_thresholds(double T, uint64_t theta[3]);

/* Metropolis acceptance cut points theta[k] = floor(exp(-beta*4(k+1)) * 2^32)
 * for dE = 4, 8, 12; a move with dE > 0 is accepted iff u < theta[dE/4 - 1]
 * (Sec. 2.3, the textbook Metropolis the paper compares against). */
int orc_metro_thresholds(double T, uint64_t theta[3]);

/* J = +-1 with probability 1/2 each, drawn once per sample (Sec. 2.1). J: [N*3]. */
void orc_init_couplings(int L, uint64_t seed, int64_t sample, int8_t *J);

/* Fully disordered start (Sec. 3: infinite-temperature initial condition). s: [N]. */
void orc_init_spins(int L, uint64_t seed, int64_t gid, int8_t *s);

/* H_EA = - sum over bonds J_xy s_x s_y, Eq. (Hamiltonian). */
int64_t orc_energy(int L, const int8_t *J, const int8_t *s);

/* Change of H_EA if s_x alone is flipped: dH = 2 s_x sum_y J_xy s_y (Sec. 2.3). */
int orc_delta_h(int L, const int8_t *J, const int8_t *s, int64_t site);

/* Draw every daemon of one replica afresh from Eq. (prob-daemons-walkers) at
 * temperature T for the refresh at global sweep t (Sec. 2.7). m: [N]. */
int orc_refresh(int L, uint64_t seed, int64_t gid, int64_t t, double T, uint8_t *m);

/* The elementary move, Eq. (Creutz) with the limited-capacity rule
 * Eq. (flip-OK), applied to every site of the given parity, one at a time. */
void orc_half_sweep(int L, const int8_t *J, int8_t *s, uint8_t *m, int parity);

/* One sweep in lexicographic site order (any order is allowed for a serial
 * update, Sec. 2.8); valid for odd L. */
void orc_serial_sweep(int L, const int8_t *J, int8_t *s, uint8_t *m);

/* The procedure of Sec. 2.8 with gamma = 1 daemon per spin and a fixed refresh
 * interval: for k in [0, n_sweeps): with t = *t_io + k, if t % interval == 0
 * refresh all daemons at T = schedule[k]; then the even half-sweep, then the
 * odd half-sweep (serial != 0: one lexicographic sweep instead). All S samples
 * and R replicas. J: [S][N*3], s and m: [S][R][N]. Advances *t_io by n_sweeps.
 * Returns 0, or -1 on a bad argument. */
int orc_run(int L, int S, int R, uint64_t seed, const int8_t *J, int8_t *s, uint8_t *m,
            int64_t *t_io, const double *schedule, int64_t n_sweeps, int32_t interval,
            int serial);

/* Refresh schedule of the procedure in Sec. 2.8 taken literally: daemons are
 * drawn before global sweeps t = 2^s - 1 (s = 0, 1, 2, ...). Same arguments as
 * orc_run without the interval. */
int orc_run_logrefresh(int L, int S, int R, uint64_t seed, const int8_t *J, int8_t *s,
                       uint8_t *m, int64_t *t_io, const double *schedule, int64_t n_sweeps);

/* Wandering of one family of walkers (Sec. 2.6): every site of the given parity
 * exchanges its walker with the one on its nearest neighbour in direction dir
 * (0: +x, 1: +y, 2: +z, 3: -x, 4: -y, 5: -z), periodic. m: [N], even L. */
void orc_wander(int L, uint8_t *m, int dir, int parity);

/* The procedure of Sec. 2.8 with gamma daemons or walkers per spin. A timestep is
 * gamma sweeps; sweep alpha uses daemon alpha (even sites, then odd sites).
 * With walkers != 0 every timestep ends with the wandering step of parity
 * t & 1 for each family alpha, direction alpha mod 6 in the order +x, +y, +z,
 * -x, -y, -z (the table of Sec. 2.8). Refresh before timestep t iff
 * t % interval == 0, or, for interval == 0, iff t = 2^s - 1; all gamma daemons
 * are drawn, daemon alpha with gid' = gid * gamma + alpha in the counter.
 * m: [S][R][gamma][N]; schedule[k] is the temperature of timestep k. */
int orc_run_ex(int L, int S, int R, int gamma, int walkers, uint64_t seed, const int8_t *J, int8_t *s,
               uint8_t *m, int64_t *t_io, const double *schedule, int64_t n_steps, int32_t interval);

/* Checkerboard Metropolis at T = schedule[k] for sweep k, drawing one uniform
 * per update attempt with dE > 0. Same layout as orc_run; no daemons. */
int orc_run_metropolis(int L, int S, int R, uint64_t seed, const int8_t *J, int8_t *s,
                       int64_t *t_io, const double *schedule, int64_t n_sweeps, int serial);

/* energy[S*R] = H_EA, aux[S*R] = H_aux = sum of n = 4 m (Sec. 2.2),
 * overlap[S*R(R-1)/2] = sum_x s^a_x s^b_x for pairs a < b in lexicographic
 * order (Sec. 3 and App. C). Any output pointer may be NULL. */
void orc_measure(int L, int S, int R, const int8_t *J, const int8_t *s, const uint8_t *m,
                 int64_t *energy, int64_t *aux, int64_t *overlap);

/* Four-point correlation of Sec. 3, exact integer sums: for each sample,
 * G[sample*L + r] = sum over replica pairs a < b, the three axes d and all
 * sites x of q_x q_{x + r e_d}, q_x = s^a_x s^b_x, periodic, r = 0 .. L-1.
 * C4(r) = G / (3 N R(R-1)/2). Requires R >= 2. */
int orc_correlation(int L, int S, int R, const int8_t *s, int64_t *G);

/* Exact enumeration of all 2^N spin states (N <= 30) by Gray code:
 * counts[E + 3N] = number of states with H_EA = E (density of states). */
int orc_enumerate_dos(int L, const int8_t *J, int64_t *counts);

/* H_EA of every one of the 2^N states (N <= 24); bit i of the state index is
 * set <=> s_i = -1. */
int orc_all_energies(int L, const int8_t *J, int64_t *E);

/* Exact one-sweep transition matrix P[a*2^N + b] (N = 8, L = 2) of MicSA with
 * every daemon drawn afresh before the sweep with probabilities pm[0..3]
 * (Sec. 2.3 and 2.7): sum over all 4^N daemon configurations. */
int orc_l2_transition_micsa(const int8_t *J, const double pm[4], double *P);

/* Exact one-sweep transition matrix of the checkerboard Metropolis sweep with
 * the quantised acceptance theta/2^32 of orc_metro_thresholds (L = 2). */
int orc_l2_transition_metro(const int8_t *J, double T, double *P);

#ifdef __cplusplus
}
#endif
#endif
