/*
 * micsa.h -- C ABI of the GB300 (sm_103a) microcanonical simulated annealing
 * library for the 3D Edwards-Anderson +-J spin glass.
 *
 * The method (Bernaschi et al., "Microcanonical simulated annealing: massively
 * parallel Monte Carlo simulations with sporadic random-number generation"):
 *   - H_EA = -sum_<x,y> J_xy s_x s_y on a periodic L^3 lattice, J = +-1 with
 *     probability 1/2 (Sec. 2.1, Eq. Hamiltonian);
 *   - one daemon per spin holding n = 4m, m in {0,1,2,3} (Sec. 2.4, 2.5);
 *   - elementary move: flip s_x and set n -> n - dH iff 0 <= n - dH <= 12
 *     (Eq. Creutz, Eq. flip-OK), even sublattice then odd sublattice (Sec. 2.8);
 *   - the only random numbers: daemons redrawn from Eq. (prob-daemons-walkers)
 *     at the annealing temperature at refresh times (Sec. 2.7).
 *
 * Conventions for every entry point:
 *   - Return MICSA_OK (0) on success or a negative MICSA_E_* code; nothing
 *     aborts. micsa_last_error() gives a message for the last failure of a
 *     handle.
 *   - Host pointers are owned by the caller and only read or written during
 *     the call; every call that returns data to the host is synchronous with
 *     respect to that data. Device memory is owned by the handle.
 *   - A handle is used by one host thread at a time.
 *   - Natural layout: site = (z*L + y)*L + x. Couplings are the three forward
 *     bonds of each site, J[(sample*N + site)*3 + d] = +-1 for the bond between
 *     site and site + e_d (d = 0: x, 1: y, 2: z), N = L^3. Spins are int8 +-1,
 *     indexed [(sample*R + replica)*N + site]; daemons the same, uint8 m in
 *     {0,1,2,3} (energy 4m).
 *   - L must be even (the checkerboard of Sec. 2.1 needs it), 2 <= L <= 1600.
 *
 * Random numbers (the paper names no generator; this is the library's
 * contract): Philox4x32-10 with key (seed mod 2^32, seed >> 32) and counters
 *   couplings: (site, 0, sample << 2 | 0, 0), word d >= 2^31 <=> J_{+d} = -1
 *   spins:     (site, 0, gid << 2 | 1, 0),    word 0 >= 2^31 <=> s = -1
 *   daemons:   (quad, t mod 2^32, gid << 2 | 2, t >> 32), u = word[lane]
 *   Metropolis:(quad, t mod 2^32, gid << 2 | 3, t >> 32), u = word[lane]
 * with gid = sample*R + replica, t the global sweep index, h = x >> 1,
 * Q = ceil(L/2 / 4), quad = ((p*L + z)*L + y)*Q + (h >> 2), lane = h & 3,
 * p = (x + y + z) & 1. A refreshed daemon is m = [u >= c0] + [u >= c1] +
 * [u >= c2] with the cut points of micsa_daemon_thresholds().
 */
#ifndef MICSA_H
#define MICSA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MICSA_OK 0
#define MICSA_E_INVALID_ARG (-1) /* bad size, odd L, T <= 0 or not finite, interval < 1 */
#define MICSA_E_OOM (-2)         /* device or host allocation failed */
#define MICSA_E_CUDA (-3)        /* a CUDA runtime call failed; see micsa_last_error */
#define MICSA_E_TIMEOUT (-4)     /* a bounded device-side wait gave up */
#define MICSA_E_BUSY (-5)        /* pool: no free slot or memory for the job now */
#define MICSA_E_NOT_FOUND (-6)   /* pool: unknown job id */
#define MICSA_E_TOO_LARGE (-7)   /* micsa_measure_noalloc: more sums than its fixed scratch holds */

/* Capacity of the fixed device scratch of micsa_measure_noalloc, in 64-bit sums. */
#define MICSA_NOALLOC_MAX_TERMS 8192

typedef struct micsa_ctx *micsa_t;

/* Allocate the state of n_samples disorder samples x n_replicas replicas of an
 * L^3 lattice on the current CUDA device; draw the couplings (Sec. 2.1) and a
 * fully disordered start (Sec. 3) from `seed`; daemons are zero until the
 * first refresh; t = 0. *out receives the handle. 1 <= n_replicas <= 128. */
int micsa_create(int L, int n_samples, int n_replicas, uint64_t seed, micsa_t *out);

/* As micsa_create with gamma (1..8) daemons per spin, or walkers if walkers != 0
 * (Sec. 2.6, 2.8): a timestep is gamma sweeps, sweep alpha uses daemon family
 * alpha, and with walkers every timestep t ends with the wandering step of
 * parity t & 1 for each family, direction alpha mod 6 in the order +x, +y, +z,
 * -x, -y, -z. micsa_run and micsa_run_logrefresh then count timesteps (t is the
 * timestep index; a refresh draws all gamma families, family alpha with Philox
 * id gid * gamma + alpha); daemons in micsa_get_state / micsa_set_state are
 * [S][R][gamma][N] and H_aux sums all families. The shared-memory engines need
 * gamma == 1 without walkers; otherwise the streaming kernel runs. */
int micsa_create_ex(int L, int n_samples, int n_replicas, int gamma, int walkers, uint64_t seed,
                    micsa_t *out);

/* Start over on the resident memory: redraw couplings and spins from `seed`
 * exactly as micsa_create does, zero the daemons, set t = 0. Asynchronous on
 * the handle's stream; no host data moves. */
int micsa_reinit(micsa_t h, uint64_t seed);

/* Replace the couplings with host J[S][N][3] of +-1 (natural layout). Spins,
 * daemons and t are kept. */
int micsa_set_couplings(micsa_t h, const int8_t *J);

/* Copy the couplings back to host J[S][N][3]. */
int micsa_get_couplings(micsa_t h, int8_t *J);

/* Run n_sweeps MicSA sweeps (Sec. 2.8, gamma = 1 daemon per spin). Sweep k
 * (k < n_sweeps) has global index t = t0 + k; if t % refresh_interval == 0 all
 * daemons are redrawn at T = schedule[k] before it (Sec. 2.7, fixed-interval
 * refresh). Each sweep updates the even sublattice, then the odd one (Eq.
 * Creutz with Eq. flip-OK). schedule is a host array of n_sweeps finite
 * temperatures > 0. t advances by n_sweeps and persists across calls, so
 * run(a) then run(b) equals run(a + b). Asynchronous on the handle's stream. */
int micsa_run(micsa_t h, const double *schedule, int64_t n_sweeps, int32_t refresh_interval);

/* As micsa_run with the refresh times of the procedure in Sec. 2.8 taken
 * literally: daemons are redrawn before global sweeps t = 2^s - 1. */
int micsa_run_logrefresh(micsa_t h, const double *schedule, int64_t n_sweeps);

/* Checkerboard Metropolis at T = schedule[k] (the random-number-greedy
 * comparison of Sec. 2.3 and App. B): a flip with dH <= 0 is accepted, one
 * with dH > 0 iff u < c(dH), c from micsa_metro_thresholds. Daemons untouched. */
int micsa_run_metropolis(micsa_t h, const double *schedule, int64_t n_sweeps);

/* Observables of the current state (Sec. 3, App. C), exact integers:
 *   energy[S*R]          H_EA per (sample, replica)
 *   aux[S*R]             H_aux = sum of daemon energies 4m
 *   overlap[S*R(R-1)/2]  sum_x s^a_x s^b_x for replica pairs a < b of each
 *                        sample, pairs in lexicographic order.
 * Host arrays; any may be NULL. Synchronous. */
int micsa_measure(micsa_t h, int64_t *energy, int64_t *aux, int64_t *overlap);

/* Four-point correlation of Sec. 3 as exact integer sums: for each sample,
 * G[sample*L + r] = sum over replica pairs a < b, the three lattice axes d and
 * all sites x of q_x q_{x + r e_d}, with q_x = s^a_x s^b_x, periodic, r = 0..L-1.
 * C4(r) = G / (3 N R(R-1)/2) (the paper's sum over a != b normalised by
 * N R(R-1)/2 counts each unordered pair once, so that C4(0) = 1). Host array
 * G[S][L]; needs R >= 2 and L <= 1024; the device scratch of the overlap
 * fields, N * S * R(R-1)/2 bytes, is limited to 4 GiB (MICSA_E_TOO_LARGE
 * beyond). Synchronous. */
int micsa_correlation(micsa_t h, int64_t *G);

/* The four-point correlation itself, C4[sample*L + r] = G[sample*L + r] /
 * (3 N R(R-1)/2) in double, G the sums of micsa_correlation (same limits and
 * errors). Host array C4[S][L]. Synchronous. */
int micsa_c4(micsa_t h, double *C4);

/* Copy the state to / from host arrays in natural layout: spins[S*R*N] int8
 * +-1, daemons[S*R*N] uint8 in {0..3}, and the global sweep index t. Any
 * pointer may be NULL (that part is skipped). set_state validates values. */
int micsa_get_state(micsa_t h, int8_t *spins, uint8_t *daemons, int64_t *t);
int micsa_set_state(micsa_t h, const int8_t *spins, const uint8_t *daemons, int64_t t);

/* Use `stream` (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream)
 * for all later work of the handle; NULL selects the handle's own stream. */
int micsa_set_stream(micsa_t h, void *stream);

/* Block until the handle's queued work is done. */
int micsa_sync(micsa_t h);

/* Device bytes held by the handle. */
int micsa_device_bytes(micsa_t h, size_t *bytes);

/* Launch shape of the sweep kernels (the autotuner's knobs; results are
 * bit-identical for every choice): words_per_thread 1, 2 or 4 (32-bit words of
 * sites per thread, reduced to what the row pitch allows), optionally ORed with
 * MICSA_LAUNCH_REGCAP for the kernel variant whose registers are capped (the
 * streaming kernel: 64 per thread, blocks of at most 128 threads, 8 per SM;
 * the bit-plane kernel: 102, 5 blocks of 128 per SM) and/or MICSA_LAUNCH_PAIRS
 * for the streaming variant in which one thread updates two neighbouring rows
 * (rows without padding, MicSA; sharing their opposite-parity rows), or
 * MICSA_LAUNCH_REPS for the streaming variant in which one thread updates its
 * words for every replica of its sample (rows without padding, MicSA; the bond
 * words and the neighbour offsets shared by the replicas), block 32..256 in
 * steps of 32 (the register-capped kernel takes at most 128 threads a block:
 * fewer replica rows per block, more blocks), blocks_per_sm -1 (grid-stride
 * loop over the resident capacity), 0 (one thread per chunk, a grid without
 * loops: the streaming kernel's fastest form at L = 160) or a positive cap,
 * pdl != 0 chains consecutive
 * half-sweeps with programmatic dependent launch, graph_sweeps > 0 replays a
 * captured CUDA graph of that many sweeps (0: direct launches). Synchronizes
 * the handle's stream. */
#define MICSA_LAUNCH_REGCAP 256
#define MICSA_LAUNCH_PAIRS 512
#define MICSA_LAUNCH_REPS 1024
int micsa_set_launch_config(micsa_t h, int words_per_thread, int block, int blocks_per_sm, int pdl,
                            int graph_sweeps);

/* Which kernel runs MicSA sweeps (results are bit-identical for every choice):
 *   MICSA_ENGINE_AUTO      MULTISPIN for L <= 32, RESIDENT for L <= 40,
 *                          STREAM above
 *   MICSA_ENGINE_STREAM    one launch per half-sweep over the lattice in HBM/L2
 *   MICSA_ENGINE_RESIDENT  each CTA keeps one replica in shared memory (bytes,
 *                          6 * L*L*P <= 200 KiB with P the row pitch, i.e.
 *                          L <= 40) for resident_sweeps sweeps per launch
 *   MICSA_ENGINE_MULTISPIN as RESIDENT with the replica held as bit planes
 *                          (32 sites per word, Boolean update; L <= 32)
 *   MICSA_ENGINE_ONCHIP    the whole state in the shared memory of all SMs:
 *                          each CTA of one cooperative launch owns a range of
 *                          (z, y) rows of one sample, exchanges the halo rows
 *                          with its neighbour CTAs through L2 and synchronizes
 *                          only with them (bounded waits), resident_sweeps
 *                          sweeps per launch. Needs gamma = 1, no walkers,
 *                          L >= 8, S <= number of SMs and a state that fits
 *                          (L = 160 with R <= 2). A wait that runs out makes
 *                          the next micsa_sync / micsa_measure /
 *                          micsa_get_state return MICSA_E_TIMEOUT.
 *   MICSA_ENGINE_TMA       as STREAM with the tiles (8 x 8 rows of a group of
 *                          two replicas, with their periodic halo rows) staged
 *                          in shared memory by TMA tensor copies into a ring
 *                          of mbarrier-tracked stages in persistent CTAs
 *                          (bounded waits, MICSA_E_TIMEOUT as ONCHIP). Needs
 *                          L % 8 == 0, a row pitch P = 4 ceil(L/8) that is a
 *                          multiple of 16 and at most 256, gamma = 1 and no
 *                          walkers.
 *   MICSA_ENGINE_MULTISPIN_GLOBAL
 *                          bit planes in HBM (32 z per word) for L a multiple
 *                          of 32: each micsa_run converts the byte state to
 *                          planes, runs one launch per half-sweep on them
 *                          (graphs, PDL) and converts back. gamma daemon
 *                          families and walkers included (the wandering step
 *                          is applied as the next timestep reads its daemons,
 *                          between two daemon buffers). Extra device memory
 *                          per spin: (2 + 4 gamma) / 16 bytes per replica,
 *                          (2 + 8 gamma) / 16 with walkers, 0.75 per sample.
 * An engine whose size limit the lattice exceeds is rejected. Runs with gamma
 * > 1 or walkers on any engine but MULTISPIN_GLOBAL use the streaming kernel;
 * Metropolis runs use it too, except on MULTISPIN_GLOBAL with gamma == 1 and no
 * walkers, where they run on the bit planes (the same Philox counters).
 * resident_sweeps only matters to RESIDENT, MULTISPIN and ONCHIP. Synchronizes.
 * (App. B and Sec. 2.5 describe the multispin Boolean update.) */
#define MICSA_ENGINE_AUTO 0
#define MICSA_ENGINE_STREAM 1
#define MICSA_ENGINE_RESIDENT 2
#define MICSA_ENGINE_MULTISPIN 3
#define MICSA_ENGINE_MULTISPIN_GLOBAL 4
#define MICSA_ENGINE_ONCHIP 5
#define MICSA_ENGINE_TMA 6
int micsa_set_engine(micsa_t h, int engine, int resident_sweeps);

/* Graph replays of the STREAM, TMA and MULTISPIN_GLOBAL engines split the replicas
 * into `chains` groups (1..4, at most n_replicas; default 1) whose half-sweeps
 * are captured as concurrent kernel chains joined at the end of each graph:
 * the groups touch disjoint replicas, so one chain's launch gaps overlap the
 * others' work. Results do not depend on it. Synchronizes. */
int micsa_set_replica_chains(micsa_t h, int chains);

/* Replicas one thread of the MULTISPIN_GLOBAL engine runs over the same bond
 * words (1 .. n_replicas; 0 = automatic: as few as keep about 2048 threads per
 * SM busy). Results do not depend on it. Synchronizes. */
int micsa_set_multispin_replicas(micsa_t h, int replicas_per_thread);

/* Self-test of the bounded wait of the ONCHIP engine: one CTA waits on an
 * epoch flag that nothing sets, giving up after `polls` polls. *timed_out
 * receives 1 when the wait ran out and reported it (the expected result).
 * Uses the current device; synchronous. */
int micsa_wait_selftest(int64_t polls, int *timed_out);

/* The engine that the next micsa_run will use (STREAM, RESIDENT, MULTISPIN,
 * MULTISPIN_GLOBAL, ONCHIP or TMA). */
int micsa_get_engine(micsa_t h, int *engine);

/* The launch shape requested (words_per_thread as set, reduced to what the row
 * pitch allows, with MICSA_LAUNCH_REGCAP if chosen). Any pointer may be NULL. */
int micsa_get_launch_config(micsa_t h, int *words_per_thread, int *block, int *blocks_per_sm,
                            int *pdl, int *graph_sweeps);

/* Number of CUDA kernels the handle has launched since it was created. */
int micsa_launch_count(micsa_t h, int64_t *count);

/* Free the handle and its device memory. NULL is allowed. */
void micsa_destroy(micsa_t h);

/* Message of the last failed call on `h` ("" if none; a static message if h is
 * NULL). Valid until the next call on h. */
const char *micsa_last_error(micsa_t h);

/* Energy, daemon energy and overlaps of caller-owned DEVICE arrays, without
 * allocating anything (the paper has no counterpart; this serves callers that
 * may not call cudaMalloc themselves or through a library: a framework whose
 * allocator must own every device byte, a serving loop that cannot take the
 * device synchronisation an allocation can cause, a fixed memory budget).
 *   spins    device int8 +-1 [S][R][N], natural layout (see above)
 *   daemons  device uint8 m in {0..3} [S][R][N], or NULL (aux is then 0)
 *   J        device int8 +-1 [S][N][3], the forward bonds of each site
 *   energy[S*R], aux[S*R], overlap[S*R(R-1)/2]  HOST arrays, as micsa_measure;
 *            any may be NULL
 *   stream   cudaStream_t to run on (NULL: the legacy default stream)
 * Limits (MICSA_E_INVALID_ARG outside them): 2 <= L <= 1600, odd L included
 * (the energy is the sum over the three forward bonds of every site, which
 * needs no checkerboard); 1 <= R <= 32; S >= 1. The sums go through one fixed
 * device array of MICSA_NOALLOC_MAX_TERMS 64-bit counters (64 KiB) that every
 * GPU loading the library holds until the process exits; a call needs
 * 2*S*R + S*R*(R-1)/2 of them and returns MICSA_E_TOO_LARGE beyond that (or
 * for S > 65535). No cudaMalloc, cudaFree or other allocating routine is
 * called. The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process, so make
 * that first call before any stream capture begins, and make no call on a
 * device after cudaDeviceReset of that device (the kept address is then
 * stale). All calls share the array (each clears what it uses first): calls
 * whose GPU work overlaps -- other streams, other host threads -- race on it.
 * Each call synchronises `stream` and returns after the host arrays are
 * written. */
int micsa_measure_noalloc(const int8_t *spins, const uint8_t *daemons, const int8_t *J, int L,
                          int n_samples, int n_replicas, int64_t *energy, int64_t *aux,
                          int64_t *overlap, void *stream);

/* ------------------------------------------------------------------------
 * Batched engine / serving pool: independent annealing jobs of mixed L,
 * replica count, length and refresh interval, resident in one device arena
 * and advanced together (one persistent launch per half-sweep over all jobs,
 * a tick of K sweeps replayed as one CUDA graph). Jobs are admitted and
 * retired between ticks (continuous batching), limited by free slots and by
 * free arena bytes. A job computes exactly what micsa_create(L, 1, R, seed)
 * followed by micsa_run(schedule, n_sweeps, refresh_interval) computes, with
 * the linear schedule T(k) = T_start + (T_end - T_start) * (k / (n_sweeps - 1))
 * in IEEE double (T(0) = T_start when n_sweeps == 1), so its result does not
 * depend on its slot or on the other jobs. After every tick (every K sweeps of
 * the job's own clock, and after its last sweep) the exact energy of each
 * replica is measured; the lowest one seen (ties: the earliest) and that
 * configuration are kept ("best configuration").
 * ------------------------------------------------------------------------ */
#define MICSA_POOL_MAX_REPLICAS 8

typedef struct micsa_pool *micsa_pool_t;

typedef struct {
    int L;                    /* even, 2..1024 */
    int n_replicas;           /* 1..MICSA_POOL_MAX_REPLICAS */
    uint64_t seed;            /* couplings, spins and daemons of this job */
    int64_t n_sweeps;         /* >= 1 */
    int32_t refresh_interval; /* >= 1 */
    double T_start, T_end;    /* finite, > 0 */
} micsa_job_desc;

typedef struct {
    int64_t job_id;
    int64_t sweeps_done;
    int32_t n_replicas;
    int64_t energy[MICSA_POOL_MAX_REPLICAS];      /* final H_EA per replica */
    int64_t aux[MICSA_POOL_MAX_REPLICAS];         /* final H_aux per replica */
    int64_t best_energy[MICSA_POOL_MAX_REPLICAS]; /* lowest H_EA at the measurement points */
    int64_t best_t[MICSA_POOL_MAX_REPLICAS];      /* sweep count where it was first seen */
} micsa_job_result;

/* Reserve an arena of arena_bytes (>= 1 MiB) on the current device and room for
 * max_jobs (1..65535) resident jobs; a tick advances every job by tick_sweeps
 * (1..4096) sweeps. */
int micsa_pool_create(size_t arena_bytes, int max_jobs, int tick_sweeps, micsa_pool_t *out);

/* Arena bytes a job needs (host-only). */
int micsa_pool_job_bytes(const micsa_job_desc *job, size_t *bytes);

/* Admit a job: returns its id in *job_id, MICSA_E_BUSY if no slot or not enough
 * contiguous arena memory is free now (retry after a completed job has been
 * polled), MICSA_E_INVALID_ARG for a bad description. Its initial state is
 * drawn on the device; nothing waits for queued ticks. */
int micsa_pool_submit(micsa_pool_t p, const micsa_job_desc *job, int64_t *job_id);

/* Queue one tick: every admitted job that is not finished advances by
 * min(tick_sweeps, sweeps left) sweeps. Asynchronous. */
int micsa_pool_tick(micsa_pool_t p);

/* Block until every queued tick has run. */
int micsa_pool_wait(micsa_pool_t p);

/* Block until at most max_pending queued ticks have not run yet (bounds how far
 * the host runs ahead of the device, so that new admissions start soon). */
int micsa_pool_wait_ticks(micsa_pool_t p, int max_pending);

/* If job `job_id` has finished and its last tick has run: fill *res, copy its
 * best configurations to best_spins[R][N] (host, natural layout, int8 +-1;
 * may be NULL), free its slot and memory, return MICSA_OK. MICSA_E_BUSY if it
 * is still running, MICSA_E_NOT_FOUND for an unknown (or already polled) id. */
int micsa_pool_poll(micsa_pool_t p, int64_t job_id, micsa_job_result *res, int8_t *best_spins);

/* micsa_pool_poll that also copies the job's final state: spins[R][N] (int8
 * +-1) and daemons[R][N] (uint8 m in {0..3}), host, natural layout, after its
 * last sweep (the state micsa_get_state of the equivalent single handle
 * returns). Either pointer may be NULL. Same return codes as micsa_pool_poll. */
int micsa_pool_poll_state(micsa_pool_t p, int64_t job_id, micsa_job_result *res, int8_t *best_spins,
                          int8_t *spins, uint8_t *daemons);

/* Ids of up to max_ids finished jobs whose last tick has run (ready to poll
 * without waiting), in *n_ids. Non-blocking. */
int micsa_pool_finished(micsa_pool_t p, int64_t *ids, int max_ids, int *n_ids);

/* Jobs resident, free arena bytes, kernels launched so far. Any pointer may be NULL. */
int micsa_pool_stats(micsa_pool_t p, int *live_jobs, size_t *free_bytes, int64_t *launches);

/* Grid of the batched kernels (blocks per SM, 1..64; 0: as many as fit, the
 * default), programmatic dependent
 * launch on/off, CUDA graph replay of ticks on/off (the autotuner's knobs;
 * results are identical for every choice). Synchronizes. */
int micsa_pool_set_launch_config(micsa_pool_t p, int blocks_per_sm, int pdl, int use_graph);

/* Shape of the streaming jobs' half-sweeps (the autotuner's other knobs;
 * results are identical for every choice): a streaming job's thread updates
 * the largest of 4, 2, 1 words (4 sites each) that is at most max_words (1, 2
 * or 4) and divides the words of its rows, for the jobs already admitted too;
 * the virtual-block table is split at (job, replica) boundaries into `chains`
 * (1..4) parts run as concurrent kernel chains. Default 4 and 2.
 * MICSA_E_INVALID_ARG otherwise. Synchronizes. */
int micsa_pool_set_shape(micsa_pool_t p, int max_words, int chains);

/* Bit-plane path for the jobs admitted from now on with L above 32 (on by
 * default): during a tick such a job's state is held as bit planes (32 sites of
 * a z column per word, the last word of a column partial when L is not a
 * multiple of 32; rows of 4 ceil(L/8) words, padded to whole Philox blocks;
 * multispin coding, App. B) and swept by the
 * bit-plane update, converted from and back to the byte layout at the tick's
 * ends; these jobs run as the same number of concurrent chains as the
 * byte-streamed ones. Results are identical either way (the same Philox
 * counters). micsa_pool_job_bytes counts the plane storage for such jobs. */
int micsa_pool_set_planes(micsa_pool_t p, int on);

/* Shared-memory path of the bit-plane jobs admitted from now on (on by
 * default, at the largest budget the device allows): a job whose replicas'
 * bit planes fit in smem_bytes of shared memory is advanced by one persistent
 * launch per tick, in units of as many replicas as fit (with its bond planes
 * when they fit too, else reading them from the arena): a CTA converts the
 * unit's bytes to planes in its shared memory, runs the tick's sweeps there
 * with the same bit-plane update and Philox counters, and converts back, so
 * the results are identical either way. smem_bytes = 0 turns it off;
 * blocks_per_sm (1..8) sets the launch's grid (CTAs of 512 threads for one per
 * SM, of 256 for more). MICSA_E_INVALID_ARG for a budget above the device's
 * limit. Synchronizes. */
int micsa_pool_set_smem_planes(micsa_pool_t p, size_t smem_bytes, int blocks_per_sm);

/* For the jobs admitted from now on (on by default): a shared-memory unit of a
 * job with 32 < L <= 128 is split over a thread-block cluster of ceil(L / 32)
 * CTAs, CTA c holding z word c (32 z) of every column of the unit's replicas;
 * the z neighbours across words are read from the peer CTAs' shared memory
 * (distributed shared memory) and a cluster barrier separates the half-sweeps,
 * so a unit's tick runs on several SMs and a replica's slice must fit the
 * budget rather than the whole replica. Off: a unit in one CTA. Results are
 * identical either way. */
int micsa_pool_set_smem_clusters(micsa_pool_t p, int on);

/* For the jobs admitted from now on (off by default): a job with L <= 32 is
 * advanced as bit planes in shared memory too, in units of as many of its
 * replicas as fit 48 KB beside its bond planes, by a persistent launch of CTAs of
 * 128 threads (four per SM) per tick; off: the shared-memory multispin kernel
 * (one replica per CTA, one thread per plane word), which measured twice as fast
 * on such lattices (a unit's word groups of four are few: 32 at L = 16). Results
 * are identical either way. */
int micsa_pool_set_small_planes(micsa_pool_t p, int on);

/* The current budget, the largest the device allows, and the blocks per SM of
 * the shared-memory bit-plane path. Any pointer may be NULL. */
int micsa_pool_get_smem_planes(micsa_pool_t p, size_t *smem_bytes, size_t *max_smem_bytes, int *blocks_per_sm);

/* Message of the last failure on p. */
const char *micsa_pool_last_error(micsa_pool_t p);

/* Free the pool and its arena (NULL allowed). */
void micsa_pool_destroy(micsa_pool_t p);

/* Cut points of the daemon refresh at temperature T, Eq. (prob-daemons-walkers):
 * with beta = 1/T, x = exp(-4 beta), p0 = (1 - x)/(1 - x^4) (x^4 as
 * (x*x)*(x*x); p0 = 1/4 when x == 1), p1 = p0 x, p2 = p1 x, c0 = p0,
 * c1 = c0 + p1, c2 = c1 + p2 in IEEE double, theta_k = min(floor(c_k 2^32), 2^32).
 * Host-only; needs no GPU. */
int micsa_daemon_thresholds(double T, uint64_t theta[3]);

/* Metropolis cut points theta_k = floor(exp(-beta*4(k+1)) 2^32), k = 0, 1, 2
 * (dH = 4, 8, 12). Host-only. */
int micsa_metro_thresholds(double T, uint64_t theta[3]);

#ifdef __cplusplus
}
#endif
#endif
