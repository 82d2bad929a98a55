/*
 * o2pic — C ABI of the GB300 (sm_103a) particle loop of the 1D3V PIC-MCC
 * model of a capacitively coupled RF oxygen discharge.
 *
 * Method: F. X. Bronold et al., "Particle-based modeling of oxygen
 * discharges", 28th ICPIG (2007), Sec. 2 (model), Table 1 (reactions),
 * Eq. 1 (associative detachment).  One call of o2pic_step advances the
 * discharge by whole time steps; each step is
 *   field gather -> leapfrog push in x (v_x, v_y, v_z carried) ->
 *   absorbing electrodes -> null-collision Monte Carlo against the O2
 *   background (n = p/kT, T_gas = 300 K) and O2(a1Dg) at C n_O2 ->
 *   births / removals -> (ion steps) cell-binned O- + O2+ neutralization (17)
 *   -> CIC charge deposition -> Poisson solve with phi(0) = U sin(2 pi f t),
 *   phi(L) = 0 -> cycle-accumulated density moments.
 *
 * Conventions for every function:
 *   - return 0 (O2PIC_OK) or a negative O2PIC_E_* code; o2pic_strerror()
 *     names it;
 *   - SI units; energies of cross-section tables in eV;
 *   - the context owns all device memory it allocates; pointers passed in are
 *     borrowed for the duration of the call only (the call copies);
 *   - `stream` is a cudaStream_t passed as void* (NULL = the context's own
 *     stream); HOST pointers may be pageable or pinned; DEVICE pointers must
 *     live on the context's device;
 *   - species index: 0 = e, 1 = O-, 2 = O2+.
 *   - work is enqueued asynchronously on the context's stream; device-side
 *     errors (capacity overflow, id overflow, non-finite particles, a bounded
 *     wait that gave up) are latched in the context and returned by the next
 *     synchronizing call (o2pic_synchronize, o2pic_read_*, o2pic_get_stats).
 *     After an error the particle state is unspecified; reload particles.
 */
#ifndef O2PIC_H
#define O2PIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define O2PIC_NSPECIES 3
#define O2PIC_MAXPROC 16

enum { O2PIC_E = 0, O2PIC_OM = 1, O2PIC_OP = 2 };

/* Process kinds (Table 1 of the paper):
 *   ELASTIC    (7), (8): isotropic; electrons in the lab frame off a target at
 *              rest with recoil loss 2m/M (1 - cos chi), ions in the CM frame
 *   EXCITE     (10)-(15): electron loses threshold_eV, isotropic
 *   IONIZE     (21): e + O2 -> 2e + O2+, the excess energy split uniformly
 *   ATTACH     (18): e + O2 -> O + O-
 *   DETACH     (19), (20): O- + O2 / O2(a) -> ... + e
 *   CX         (9): O2+ + O2 charge exchange (ion takes the target velocity)
 *   NEUTRALIZE (17): O- + O2+ -> neutrals, binary, cell-local (give it with
 *              species O-, target ION; sigma is the neutralization cross
 *              section, e.g. the Landau-Zener form of the paper)
 *   RECOMBINE  (16): e + O2+ -> O + O, binary and cell-local like (17), on
 *              ion steps before (17) (species e, target ION)
 *   EDETACH    (22): e + O- -> O + 2e, binary and cell-local like (17), on
 *              ion steps before (16) and (17) (species O-, target ELECTRON;
 *              threshold_eV = the O electron affinity): the O- is removed,
 *              the electron loses the threshold and shares the rest uniformly
 *              with the detached electron, both isotropic about the O-'s
 *              velocity; the newborn, at the O-'s place, follows the step's
 *              other electron births in the order of the O- parents */
enum { O2PIC_ELASTIC = 0, O2PIC_EXCITE = 1, O2PIC_IONIZE = 2, O2PIC_ATTACH = 3,
       O2PIC_DETACH = 4, O2PIC_CX = 5, O2PIC_NEUTRALIZE = 6, O2PIC_RECOMBINE = 7, O2PIC_EDETACH = 8 };

/* Targets: ground-state O2 (density p/kT), metastable O2(a1Dg) (density
 * C_meta p/kT, Sec. 2), the other ion species ((16), (17)) or the electrons
 * ((22)). */
enum { O2PIC_TARGET_O2 = 0, O2PIC_TARGET_O2_META = 1, O2PIC_TARGET_ION = 2, O2PIC_TARGET_ELECTRON = 3 };

enum { O2PIC_HOST = 0, O2PIC_DEVICE = 1 };

#define O2PIC_OK 0
#define O2PIC_E_INVALID_ARG (-1)
#define O2PIC_E_CAPACITY (-2)
#define O2PIC_E_ID_OVERFLOW (-3)
#define O2PIC_E_NONFINITE (-4)
#define O2PIC_E_CUDA (-5)
#define O2PIC_E_TIMEOUT (-6)
#define O2PIC_E_STATE (-7)

typedef struct o2pic_ctx o2pic_ctx;

/* Discharge configuration (Sec. 2): gap L [m], RF frequency f [Hz], voltage
 * amplitude U [V] on the electrode at x = 0 (the one at x = L is grounded),
 * pressure p [Pa], gas temperature T_gas [K] (300 in the paper), metastable
 * fraction C_meta (n_Delta = C n_O2), time step dt [s], macro-particle weight
 * [particles per m^2 of electrode], electrode area [m^2], masses [kg],
 * n_cells grid cells (n_cells + 1 nodes), ions pushed every ion_subcycle
 * steps with dt_ion = ion_subcycle dt, seed of the Philox streams,
 * capacity[s] = maximum particles of species s (live + dead slots + births
 * of one step), compact_check = steps between checks for dead slots
 * (0 = default 16), device = CUDA ordinal. */
typedef struct {
    double L, f, U, p, T_gas, C_meta, dt, weight, area;
    double m_e, m_OM, m_OP, M_gas;
    int32_t n_cells, ion_subcycle;
    uint32_t seed, compact_check;
    uint64_t capacity[O2PIC_NSPECIES];
    int32_t device, reserved;
} o2pic_config;

/* One cross-section table: sigma_m2[i] at E_eV[i] (n >= 1, E strictly
 * increasing), linearly interpolated, constant beyond the ends, zero below
 * threshold_eV. */
typedef struct {
    int32_t species, kind, target, n;
    double threshold_eV;
    const double* E_eV;
    const double* sigma_m2;
} o2pic_process;

/* Counters since create (or the last load of all species); layout is fixed. */
typedef struct {
    uint64_t events[O2PIC_NSPECIES][O2PIC_MAXPROC]; /* real collisions per process */
    uint64_t absorbed[O2PIC_NSPECIES][2];           /* [species][0: x<0, 1: x>=L] */
    uint64_t born[O2PIC_NSPECIES];
    uint64_t neutralized, pair_candidates, particle_steps;
    uint64_t warn_emax;      /* energy above the 2^12 eV table grid */
    uint64_t warn_tries;     /* a rejection loop hit its cap */
    uint64_t warn_pair_gt1;  /* neutralization probability above 1 */
    uint64_t id_overflow;
    uint64_t step;
    uint64_t live[O2PIC_NSPECIES];
    uint64_t slots[O2PIC_NSPECIES];
    uint64_t next_id[O2PIC_NSPECIES];
    uint64_t error_flags;
    uint64_t particle_steps_species[O2PIC_NSPECIES];  /* particles pushed, per species */
    uint64_t recombined, rec_candidates;              /* (16): pairs removed, pairs tested */
    uint64_t edetached, edet_candidates;              /* (22): pairs reacted, pairs tested */
    uint64_t coulomb_pairs;                           /* (1)-(6): pairs scattered */
    uint64_t warn_numax;     /* candidates whose total rate exceeded a capped nu_max */
} o2pic_stats;

/* Fills `cfg` with the defaults (parity-case geometry, T_gas = 300 K, O, O2
 * masses, capacity 0 = must be set). */
int o2pic_config_init(o2pic_config* cfg);

/* Validates `cfg`, selects the device, allocates all device memory
 * (particles: 2 x 20 B x capacity per species) and returns a context in *out.
 * Errors: INVALID_ARG (bad configuration; no CUDA call is made), CUDA. */
int o2pic_create(const o2pic_config* cfg, o2pic_ctx** out);

/* Builds the per-species rate tables nu_k(E_i) = n_target sigma_k(E_i) g(E_i)
 * on 32 points per octave over [2^-10, 2^12] eV (FP64, stored FP32 as
 * cumulative sums), nu_max and P_max = 1 - exp(-nu_max dt_s) (null-collision
 * method, Sec. 2), and the rate-coefficient tables of the binary processes
 * (17), (16), (22); copies them to the device.  At most O2PIC_MAXPROC
 * processes per species, one NEUTRALIZE, one RECOMBINE, one EDETACH.
 * Errors: INVALID_ARG. */
int o2pic_set_processes(o2pic_ctx* ctx, const o2pic_process* procs, int nproc);

/* Majorant caps of the null-collision method (Sec. 2), per species in eV,
 * taking effect at the next o2pic_set_processes: nu_max = the largest total
 * rate nu(E_i) over the grid points up to the first one at or above the cap,
 * instead of over the whole grid (NaN or +inf: the whole grid, the default).
 * A cap is a bound on the energies the species reaches (for ions, the
 * relative energy stays below the applied voltage's energy); a candidate
 * whose total rate exceeds nu_max collides with probability 1 instead of
 * nu(E) / nu_max and is counted in o2pic_stats.warn_numax, which is 0 when
 * the cap holds.  `cap_eV` is a host array of O2PIC_NSPECIES doubles, read
 * during the call.  Errors: INVALID_ARG (a cap that is not positive). */
int o2pic_set_majorant_cap(o2pic_ctx* ctx, const double* cap_eV);

/* Coulomb elastic collisions (1)-(6) of Table 1: e-e, O- - O-, O2+ - O2+,
 * e - O2+, e - O-, O- - O2+; bit r-1 of `mask` enables reaction r (0 = off,
 * the default).  Model: the binary collisions of Takizuka & Abe (J. Comput.
 * Phys. 25, 205, 1977) with the Coulomb logarithm ln_lambda: on ion steps,
 * with dt_ion, after the species' pushes and collisions and before the
 * reactive pairs, within each cell each pair's relative velocity turns by
 * theta, tan(theta/2) ~ N(0, sigma^2), sigma^2 = q_a^2 q_b^2 n lnL dt_ion /
 * (8 pi eps0^2 mu^2 g^3) (n: the species' density for like pairs, the larger
 * density for unlike pairs, paired min(n_a, n_b) times), azimuth uniform;
 * each pair keeps its momentum and energy.  Errors: INVALID_ARG, CUDA. */
int o2pic_set_coulomb(o2pic_ctx* ctx, uint32_t mask, double ln_lambda);

/* Replaces species `species` by n particles (SoA float32 x, vx, vy, vz and
 * uint32 ids, unique within the species); velocities are taken as
 * v^{n-1/2}.  mem_kind = O2PIC_HOST or O2PIC_DEVICE.  The next step starts
 * with a fresh deposit and field solve.  New ids continue at max(id) + 1.
 * The particles are checked on the device after the copy; on INVALID_ARG
 * (x outside [0, L) or a non-finite velocity) the species is left empty.
 * Errors: INVALID_ARG (also n > capacity, no copy made), CUDA. */
int o2pic_load_particles(o2pic_ctx* ctx, int species, const float* x, const float* vx,
                         const float* vy, const float* vz, const uint32_t* id, uint64_t n,
                         int mem_kind, void* stream);

/* Free flights (Sec. 2: the durations of the free flights between
 * collisions follow from kinetic considerations).  Each particle carries the
 * step at which its current free flight ends: its next null-collision
 * candidate (low 32 bits of the step index).  A flight of K pushes,
 * K ~ Geometric(P_max) (the same law as a Bernoulli(P_max) test at every
 * push), is drawn from the particle's random stream when the particle is
 * loaded or born and at each of its candidates.  Loaded particles get fresh
 * flights, drawn at the first step after the load (or new tables); to resume
 * a saved run bit for bit, save them with o2pic_read_flight and restore them
 * with o2pic_load_flight right after o2pic_load_particles (and set the saved
 * step with o2pic_set_step).
 *
 * o2pic_load_flight: tc[0..n) for the particles just loaded into `species`
 * (n must equal the loaded count; HOST or DEVICE memory).
 * o2pic_read_flight: the flights of the live particles of `species` in array
 * order (the order of o2pic_read_particles), up to cap; *n = live count.
 * Errors: INVALID_ARG, CUDA. */
int o2pic_load_flight(o2pic_ctx* ctx, int species, const uint32_t* tc, uint64_t n, int mem_kind, void* stream);
int o2pic_read_flight(o2pic_ctx* ctx, int species, uint32_t* tc, uint64_t cap, uint64_t* n, int mem_kind);

/* Sets the id the next particle born in `species` gets (it must exceed every
 * id of that species): with o2pic_set_step and the particles of a saved state
 * (o2pic_read_particles, o2pic_get_stats().next_id and .step) a run resumes
 * bit for bit.  Ids are 32-bit: a birth whose id would reach 2^32 sets
 * O2PIC_E_ID_OVERFLOW (counted per birth in o2pic_stats.id_overflow; the
 * particle keeps the low 32 bits of its id).
 * Errors: INVALID_ARG (also next_id below the current next id, e.g. below
 * the largest loaded id + 1), CUDA. */
int o2pic_set_next_id(o2pic_ctx* ctx, int species, uint32_t next_id);

/* Enqueues nsteps time steps (Sec. 2 loop; see the file header) on `stream`.
 * Asynchronous; errors of the enqueued work appear at the next sync. */
int o2pic_step(o2pic_ctx* ctx, uint64_t nsteps, void* stream);

/* Waits for the context's work and returns the first latched error. */
int o2pic_synchronize(o2pic_ctx* ctx);

/* Live particles of `species` in array order (the order the method defines:
 * survivors in order, then births in creation order), up to `cap`; *n gets
 * the live count (even when it exceeds cap).  mem_kind as for load. */
int o2pic_read_particles(o2pic_ctx* ctx, int species, float* x, float* vx, float* vy, float* vz,
                         uint32_t* id, uint64_t cap, uint64_t* n, int mem_kind);

/* Current field on the n_cells + 1 nodes: phi [V] (FP64) and E [V/m] (the
 * FP32 copy the gather uses); either pointer may be NULL.  Host memory. */
int o2pic_read_field(o2pic_ctx* ctx, double* phi, float* E);

/* Current densities through the gap (Fig. 5 of the paper) of the steps
 * first_step .. first_step+n-1, out[5 i + k] [A/m^2]:
 *   k = 0, 1, 2: conduction current of e, O-, O2+, gap-averaged,
 *                J_s = q_s w sum_p v_x,p^{n+1/2} / (A L) over the particles
 *                pushed in the step (the ions' last push on steps without
 *                one), summed exactly in fixed point (trunc(256 v_x));
 *   k = 3: displacement current eps0 (V(t^{n+1}) - V(t^n)) / (L dt) of the
 *          prescribed electrode voltage V = U sin(2 pi f t) (the gap
 *          average of eps0 dE/dt);
 *   k = 4: total current density (k = 0..3 summed), uniform across the gap.
 * The device keeps the last 8191 completed steps since the last load or
 * set_step; steps outside that window return INVALID_ARG.  Host memory. */
int o2pic_read_currents(o2pic_ctx* ctx, uint64_t first_step, uint64_t n, double* out);

/* Fixed-point node charges (2^16 per macro-particle, CIC) of the current
 * particles, Q[3][n_cells+1], and their sum over the steps since the last
 * reset, Qacc[3][n_cells+1] (either may be NULL); *acc_steps = steps summed.
 * Host memory. */
int o2pic_read_charge(o2pic_ctx* ctx, uint64_t* Q, uint64_t* Qacc, uint64_t* acc_steps);

/* Cycle-averaged densities (Figs. 3-4 of the paper) [m^-3] on the nodes,
 * density[3][n_cells+1], from the accumulated charge (wall nodes hold half a
 * cell); reset != 0 restarts the accumulation.  Host memory. */
int o2pic_read_moments(o2pic_ctx* ctx, double* density, uint64_t* acc_steps, int reset);

int o2pic_get_stats(o2pic_ctx* ctx, o2pic_stats* out);

/* Sets the step counter (the RNG streams are keyed by it): with the
 * particles of a saved state this resumes a run bit for bit. */
int o2pic_set_step(o2pic_ctx* ctx, uint64_t step);

/* Kernel timing with CUDA events on the launching stream: on != 0 records an
 * event pair around every launch; o2pic_get_timing returns, per kernel kind
 * (0 push e, 1 push O-, 2 push O2+, 3 pair histograms, 4 pair, 5 field,
 * 6 compact, 7 deposit, 8 collisions e, 9 collisions O-, 10 collisions O2+,
 * 11 (16), (22) pairing, 12 candidate filter O-, 13 candidate filter O2+,
 * 14 Coulomb collisions (cell sort and reactions)),
 * the summed milliseconds and launches; items is reserved (zeros). */
int o2pic_set_timing(o2pic_ctx* ctx, int on);
int o2pic_get_timing(o2pic_ctx* ctx, double* ms, uint64_t* launches, uint64_t* items, int nkinds);

/* Kernels launched by this context since create. */
uint64_t o2pic_launch_count(o2pic_ctx* ctx);

/* The library's random streams: out[4i..4i+3] = Philox4x32-10(ctr[4i..],
 * key[2i..]) (Salmon et al., SC'11).  Device pointers, n <= 2^31. */
int o2pic_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, uint64_t n, void* stream);

/* The single-precision log used by the polar normal method (atanh series),
 * out[i] = ln(x[i]) for x in (0, 1].  Device pointers. */
int o2pic_ln_f32(const float* x, float* out, uint64_t n, void* stream);

/* Stable compaction of a caller's particle arrays (the removal part of the
 * step's births/removal, e.g. of particles absorbed at the electrodes or
 * consumed by attachment, detachment or neutralization): the particles whose
 * x is NaN (the library's marker of a removed particle) are dropped, the
 * others are written to ox.. oid in their input order.  All pointers are
 * device pointers of the current device; outputs hold n elements and must
 * not overlap the inputs; *n_out (device) receives the number kept.  The call
 * allocates its scratch (tile look-back state, 24 B per 8192 particles) with
 * cudaMalloc, frees it, and returns once the work on `stream` is done.
 * n <= 2^31.  Errors: INVALID_ARG, CUDA, TIMEOUT. */
int o2pic_compact_particles(const float* x, const float* vx, const float* vy, const float* vz,
                            const uint32_t* id, uint64_t n, float* ox, float* ovx, float* ovy, float* ovz,
                            uint32_t* oid, uint64_t* n_out, void* stream);

/* Failure detection of the bounded device waits: runs the decoupled
 * look-back wait that the compaction kernels use (one thread waiting, as tile
 * 1, for a tile 0 whose flag nothing ever sets) on `stream`.  The wait must
 * give up after its spin limit, record the timeout and return, so that the
 * context stays usable; *seconds (may be NULL) gets the kernel's duration.
 * Returns O2PIC_E_TIMEOUT when the wait gave up as designed, O2PIC_OK if it
 * did not (never expected), CUDA on a CUDA error.  No counterpart in the
 * paper: this is a property of the library. */
int o2pic_check_bounded_wait(double* seconds, void* stream);

/* The same compaction for callers that cannot allocate device memory when
 * they need it: a framework whose caching allocator already holds the free
 * memory of the device, or a pipeline that cannot accept the synchronization
 * that cudaFree brings.  No counterpart in the paper: this is a property of
 * the library, not of the method.  Arguments, results and errors as for
 * o2pic_compact_particles, except that it calls no allocator: its scratch is
 * a static device array sized for at most O2PIC_NOALLOC_MAX_PARTICLES
 * particles (about 96 KB, held on every GPU that loads the library until the
 * process exits); n beyond that returns INVALID_ARG.  Every call looks up the
 * array's device address on the current device (which must be the device of
 * the pointers).  The call copies its error word back and synchronizes
 * `stream` before it returns.  All calls on a device share the array, so
 * calls whose GPU work overlaps (e.g. on two streams at once) race: serialize
 * them.  The call resets what must start at zero itself. */
#define O2PIC_NOALLOC_MAX_PARTICLES (1ull << 25)
int o2pic_compact_particles_noalloc(const float* x, const float* vx, const float* vy, const float* vz,
                                    const uint32_t* id, uint64_t n, float* ox, float* ovx, float* ovy, float* ovz,
                                    uint32_t* oid, uint64_t* n_out, void* stream);

/* ---- Launch shape and batched stepping (many discharges, one graph) ----
 *
 * A parameter sweep (voltages, pressures, particle counts) runs many small
 * discharges; each is one context.  A batch advances all of them together
 * with one CUDA graph of steps_per_launch time steps.  When the contexts
 * share the step schedule (ion subcycle, compaction period and their phase)
 * the graph holds one batched launch per kernel and step for all of them:
 * each block of a batched grid works for one discharge (a block map), so a
 * sweep of small discharges needs a handful of launches per step instead of
 * a handful per discharge.  Otherwise (or with the environment variable
 * O2PIC_BATCH_BRANCHES=1) each context gets its own graph branch.  The
 * method is unchanged: every context gives exactly the results of
 * o2pic_step, whatever the batch, the mode and the launch shape. */

/* Blocks of the particle kernels (push and collisions) per species, in
 * [max(1, capacity / 2^23), 8 * SMs] (a block's shared-memory deposit counts
 * fewer than 2^24 particles per cell); results do not depend on them.
 * Defaults (set by o2pic_set_processes): as many as fit the GPU at once. */
int o2pic_set_launch_shape(o2pic_ctx* ctx, const int32_t push_blocks[3]);
int o2pic_get_launch_shape(o2pic_ctx* ctx, int32_t push_blocks[3]);

typedef struct o2pic_batch o2pic_batch;   /* opaque, library-owned */

/* Captures the graph.  ctxs: n >= 1 contexts on one device, each with
 * processes set and particles loaded (borrowed: they must outlive the batch
 * and are not to be stepped alone while it exists).  steps_per_launch in
 * [1, 2048], a multiple of every context's ion_subcycle and compact_check.
 * Errors: INVALID_ARG, STATE (a context without tables), CUDA. */
int o2pic_batch_create(o2pic_ctx* const* ctxs, int32_t n, uint64_t steps_per_launch, o2pic_batch** out);

/* Enqueues `launches` replays of the graph (launches * steps_per_launch
 * steps of every context) on the batch's own stream; asynchronous. */
int o2pic_batch_step(o2pic_batch* b, uint64_t launches);

/* The batch's own CUDA stream (cudaStream_t), on which o2pic_batch_step
 * enqueues its work: a caller may record events on it to time replays. */
void* o2pic_batch_stream(o2pic_batch* b);

/* Waits for the batch and returns the first error latched by any context. */
int o2pic_batch_synchronize(o2pic_batch* b);

/* Autotuner: tries launch-shape policies (particle-kernel blocks from a
 * target number of particles per warp, and the default full-GPU shape),
 * times one graph replay of each on the real batch (these replays are real
 * steps of the discharges: 7 policies x steps_per_launch steps, plus one
 * replay of the other launch mode when the contexts share their schedule),
 * keeps the fastest shape and mode and re-captures the graph.  The shapes
 * stay set on the contexts, so a batch created afterwards with another
 * steps_per_launch uses them. */
#define O2PIC_TUNE_MAX 8
typedef struct {
    int32_t n;                                   /* policies tried */
    int32_t particles_per_warp[O2PIC_TUNE_MAX];  /* 0 = default full-GPU shape */
    double ms[O2PIC_TUNE_MAX];                   /* one replay, CUDA events */
    int32_t chosen;                              /* index of the policy kept */
    int32_t fused;                               /* 1: batched launches kept, 0: one branch per context */
    double other_mode_ms;                        /* the other mode at the chosen shape (0: not tried) */
} o2pic_tune_report;
int o2pic_batch_autotune(o2pic_batch* b, o2pic_tune_report* report);

void o2pic_batch_destroy(o2pic_batch* b);

/* ---- Learned warm start: a small MLP trained on converged runs ----------
 *
 * Maps normalized discharge parameters (U, p, L, C) to cycle-averaged
 * log-density profiles; the profiles load the initial particles of a new run
 * so that it needs fewer RF cycles to converge.  No counterpart in the
 * paper.  widths[0] inputs ... widths[n-1] outputs (2 <= n <= 16, each in
 * [1, 8192]); tanh on hidden layers, linear output, bf16 weights with an fp32
 * master copy, fp32 accumulation, deterministic results.  Parameters
 * (host, fp32): for each layer W[in][out] row-major, then b[out].  Initial
 * weights Glorot-uniform from SplitMix64(seed), biases 0.  X, Y, T, grad and
 * loss are device pointers; X [B][in], Y and T [B][out] row-major. */
typedef struct o2pic_mlp o2pic_mlp;
int o2pic_mlp_create(const int32_t* widths, int32_t n_widths, uint64_t seed, o2pic_mlp** out);
uint64_t o2pic_mlp_num_params(o2pic_mlp* m);
int o2pic_mlp_set_params(o2pic_mlp* m, const float* host_params);   /* also resets the Adam state */
int o2pic_mlp_get_params(o2pic_mlp* m, float* host_params);
int o2pic_mlp_forward(o2pic_mlp* m, const float* X, float* Y, int32_t B, void* stream);
/* loss = mean over B x out of (Y - T)^2; grad (may be NULL) = its gradient
 * in the parameter layout. */
int o2pic_mlp_gradients(o2pic_mlp* m, const float* X, const float* T, int32_t B, float* grad, float* loss,
                        void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the same loss. */
int o2pic_mlp_train_step(o2pic_mlp* m, const float* X, const float* T, int32_t B, float lr, float* loss,
                         void* stream);
void o2pic_mlp_destroy(o2pic_mlp* m);

const char* o2pic_strerror(int code);

void o2pic_destroy(o2pic_ctx* ctx);

int o2pic_version(void);

#ifdef __cplusplus
}
#endif

#endif /* O2PIC_H */
