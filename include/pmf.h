/*
 * pmf.h -- C ABI of the GB300 (sm_103a) parallel step-wise pulling library.
 *
 * The library computes free-energy differences with the parallel pulling
 * protocol (PPP) of Ngo, "A Parallel-pulling Protocol for Free Energy
 * Evaluation" (arXiv 1105.4840): s independent restrained simulations, one
 * per window lambda_1..lambda_s, each started from the same state x_o and
 * relaxed for tau_i (Sec. III (ii)); the recorded reaction-coordinate
 * samples x_i give the step-wise work of Eq. (9), the Jarzynski estimate of
 * Eq. (12), the Gaussian estimate of Eq. (13), the alternative formula of
 * Eq. (14) and their combination (Sec. IV B, Sec. V).
 *
 * Conventions
 *   - Every call returns a pmf_status; no C++ exception crosses the ABI.
 *     On failure pmf_last_error() returns a thread-local message.
 *   - Input arrays are host pointers unless stated, read during the call and
 *     copied; the caller keeps ownership.  Output buffers are caller-owned
 *     host memory unless stated.
 *   - Handles are not thread-safe; use one handle per thread or lock.
 *   - All GPU work runs on the library stream (pmf_set_stream); calls that
 *     return host results synchronise that stream.
 *   - There is no CPU fallback: without a CUDA device every compute call
 *     fails with PMF_ECUDA.
 */
#ifndef PMF_H
#define PMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PMF_OK = 0,
    PMF_EINVAL = 1,   /* bad argument (sizes, monotone lambda, capacity ...)   */
    PMF_ENOMEM = 2,   /* device or host allocation failed                      */
    PMF_ECUDA = 3,    /* CUDA runtime error or no device                       */
    PMF_ENUMERIC = 4, /* a trajectory became non-finite (device error flag)    */
    PMF_ETIMEOUT = 5, /* the run exceeded pmf_run_params.timeout_s, or a device
                         wait exceeded pmf_run_params.segment_wait_s           */
    PMF_ESTATE = 6    /* call out of order (e.g. results of an unfinished run) */
} pmf_status;

enum { PMF_MODEL_1D_DOUBLEWELL = 0, PMF_MODEL_CHAIN = 1 };
enum { PMF_FP32 = 0, PMF_FP64 = 1 };

typedef struct pmf_system pmf_system; /* opaque; device copy of the system    */
typedef struct pmf_run pmf_run;       /* opaque; device x samples of one run  */

/*
 * System description: H_o of Sec. II plus the trap on the reaction
 * coordinate x (Eq. (3)).  For PMF_MODEL_CHAIN, x = |r_{N-1} - r_0| (the
 * end-to-end distance of a bead chain standing in for the deca-alanine of
 * Sec. IV) and
 *   H_o = sum_bonds bond_k/2 (r - bond_r0)^2
 *       + sum_angles angle_k/2 (theta - angle_theta0)^2
 *       + sum_dihedrals sum_{n=1..3} K_n [1 + cos(n phi - delta_n)]
 *       + sum_{|i-j|>=3} 4 eps_ij [(s_ij/r)^12 - (s_ij/r)^6] + coulomb_k q_i q_j / r
 * with s_ij = (sigma_i + sigma_j)/2 and eps_ij = sqrt(eps_i eps_j).
 * For PMF_MODEL_1D_DOUBLEWELL, H_o = dw_a (x^2 - 1)^2 in units of kT.
 */
typedef struct {
    int model;                  /* PMF_MODEL_*                                   */
    int precision;              /* chain integration: PMF_FP32 or PMF_FP64       */
    /* chain model (concatenated over chains; bead b of chain c is row
       offset_c + b with offset_c = sum of n_beads of the chains before c)     */
    int n_chains;               /* >= 1                                          */
    const int *n_beads;         /* [n_chains], each 4 .. 1024                    */
    const double *sigma;        /* [sum n_beads] nm                              */
    const double *epsilon;      /* [sum n_beads] kJ/mol (>= 0)                   */
    const double *charge;       /* [sum n_beads] e                               */
    const double *mass;         /* [sum n_beads] amu (> 0)                       */
    const double *dih_k;        /* [sum n_beads][3] K_1..K_3 of the dihedral
                                   starting at that bead (ignored for the last 3) */
    const double *dih_phase;    /* [sum n_beads][3] delta_n, each 0 or pi        */
    const double *pos0;         /* [sum n_beads][3] start state x_o (nm)         */
    double bond_k, bond_r0;     /* kJ/mol/nm^2, nm                               */
    double angle_k;             /* kJ/mol/rad^2 (0 disables angles)              */
    double angle_theta0;        /* rad                                           */
    double coulomb_k;           /* kJ mol^-1 nm e^-2                             */
    int nonbonded;              /* 0 disables the LJ and Coulomb terms           */
    /* 1D model */
    double dw_a;                /* U(x) = dw_a (x^2 - 1)^2                       */
    double x0;                  /* start state x_o                               */
} pmf_system_desc;

/* Build the device copy of a system.  *out receives a library-owned handle
 * (free with pmf_destroy_system).  PMF_EINVAL on inconsistent sizes or
 * values; PMF_ECUDA without a device. */
pmf_status pmf_create_system(const pmf_system_desc *desc, pmf_system **out);
void pmf_destroy_system(pmf_system *sys);

/*
 * Run parameters: the paper's problem statement (Sec. III, Sec. IV B):
 * trap stiffness k, temperature (as kT), relaxation time per window
 * (n_steps * dt, or n_steps_per_window[i] * dt), plus the sampling of x
 * (Sec. IV A: x recorded every 0.1 ps) and the Langevin settings.
 * Chain: BAOAB Langevin with friction gamma (1/ps).  1D: overdamped
 * Euler-Maruyama x += F dt/gamma + sqrt(2 kT dt/gamma) xi.
 * Replica uid of (window w, replica r) = uid_base + w * replicas + r; the
 * Langevin noise of a replica is Philox4x32-10 with key seed: block b of
 * counter (b, uid, step, 0) gives the normals of degrees of freedom
 * 4b..4b+3 (dof = 3 * bead + axis); initial velocities use (b, uid, 0, 1).
 */
typedef struct {
    double k;                   /* trap stiffness (energy / length^2)            */
    double kT;                  /* k_B T in the system's energy unit             */
    double dt;                  /* time step                                     */
    double gamma;               /* friction                                      */
    int64_t n_steps;            /* steps per window (used if the array is NULL)  */
    const int64_t *n_steps_per_window; /* optional [n_windows]                   */
    int64_t n_equil;            /* steps discarded before sampling; < 0: 10 %    */
    int sample_stride;          /* steps between samples (>= 1)                  */
    int replicas;               /* replicas per window (>= 1)                    */
    uint64_t seed;              /* Philox key                                    */
    uint32_t uid_base;          /* first replica uid (sharding across processes) */
    int chain;                  /* chain index of a multi-chain system           */
    double timeout_s;           /* wall-clock limit of pmf_run_wait; 0: none     */
    double segment_wait_s;      /* persistent chain launches: longest device wait
                                   for a replica's previous segment (0: 60 s,
                                   at most 1e6)                                  */
} pmf_run_params;

/* PPP of Sec. III (ii): allocate the run, upload lambda[n_windows] (strictly
 * monotone, 1 <= n_windows <= 1024), launch every window x replica simulation from
 * the system's start state x_o, and wait.  Equivalent to pmf_run_prepare +
 * pmf_run_launch + pmf_run_wait.  *out is library-owned (pmf_destroy_run);
 * it is set even when the run fails with PMF_ENUMERIC / PMF_ETIMEOUT so the
 * caller can inspect or destroy it. */
pmf_status pmf_run_windows(pmf_system *sys, const double *lambda, int n_windows,
                           const pmf_run_params *p, pmf_run **out);

/* The three phases of pmf_run_windows.  prepare allocates and uploads (the
 * only host-to-device traffic); launch enqueues the simulation on the
 * library stream and returns at once; wait blocks until it finishes and
 * reports the device error flags:
 *   PMF_ENUMERIC  a trajectory became non-finite;
 *   PMF_ETIMEOUT  a persistent chain launch waited longer than
 *                 segment_wait_s for a replica's previous segment (the
 *                 kernel raised the flag and returned by itself).
 * If timeout_s > 0 and passes first, wait raises a stop flag in host-mapped
 * memory that the persistent chain launches poll between work items, waits
 * for the kernels in flight to finish the segment they are on (1D runs and
 * one-CTA-per-replica launches run their chunk to its end), and returns
 * PMF_ETIMEOUT.  After either PMF_ETIMEOUT the run's samples are incomplete
 * and the result calls return PMF_ESTATE until a new launch finishes.
 * launch may be called again on a finished run to repeat it from x_o with
 * the same streams (identical results). */
pmf_status pmf_run_prepare(pmf_system *sys, const double *lambda, int n_windows,
                           const pmf_run_params *p, pmf_run **out);
pmf_status pmf_run_launch(pmf_run *run);

/* As pmf_run_prepare, but every replica starts from its own state instead
 * of the common x_o: start[(w * replicas + r) * N * 3 + 3 b + axis] (chain)
 * or start[w * replicas + r] (1D), host, copied.  Used to seed inserted
 * windows from stored end states (the learned window placement); the
 * paper's protocol itself starts every window from x_o (Sec. III (ii)). */
pmf_status pmf_run_prepare_seeded(pmf_system *sys, const double *lambda, int n_windows, const pmf_run_params *p,
                                  const double *start, pmf_run **out);
pmf_status pmf_run_wait(pmf_run *run);
void pmf_destroy_run(pmf_run *run);

/* Sequential pulling protocol (Sec. III (i)): each of p->replicas
 * independent simulations starts from x_o at lambda_1, relaxes p->n_steps
 * steps (tau) while x is recorded, then continues from the state reached with
 * the trap moved to lambda_2, and so on to lambda_s, in one continuous run
 * (steps numbered 0 .. s * tau - 1 for the noise; equilibration n_equil and
 * sampling count from each window's first step).  Simulation r uses uid
 * uid_base + r for every window.  The samples land in the layout of
 * pmf_run_info (window w, replica r = simulation r), so every estimator call
 * applies unchanged; pmf_final_state returns one state per simulation.
 * n_steps_per_window must be NULL; 1 <= n_windows <= 1024; s * tau < 2^32.
 * Launch, wait and the reductions as for pmf_run_prepare.  Chain runs use
 * the persistent launch (segments of at most pmf_chain_set_grid's seg_steps
 * inside each window). */
pmf_status pmf_run_prepare_sequential(pmf_system *sys, const double *lambda, int n_windows,
                                      const pmf_run_params *p, pmf_run **out);

/* Batched runs.  One pmf_batch_item is one independent PPP path (Sec. III
 * (ii)): windows lambda[n_windows] (strictly monotone) on chain `chain` of
 * the system (ignored for the 1D model).  pmf_run_batch_prepare lays the
 * items' windows end to end (item m's windows follow item m-1's; at most
 * PMF_MAX_RUN_WINDOWS in all) and shares p (p->chain is ignored; per-window
 * step counts, if given, cover the concatenated windows).  Replica uids
 * continue across items (uid_base + global window * replicas + r), so each
 * replica of the batch draws its own noise stream.  pmf_run_launch then
 * enqueues the whole batch: the launch sequence (one chain-kernel launch per
 * item per 1e5-step chunk) is captured once into a CUDA graph and replayed
 * by every later launch.  Samples and final states follow the concatenated
 * window order.  The paper runs one path at a time; batching many paths is
 * this library's addition.  Free energies per item: pmf_free_energy_item. */
typedef struct {
    int chain;                  /* chain index of the system                     */
    int n_windows;              /* >= 1                                          */
    const double *lambda;       /* host, [n_windows], copied                     */
} pmf_batch_item;
#define PMF_MAX_RUN_WINDOWS 4096
pmf_status pmf_run_batch_prepare(pmf_system *sys, const pmf_batch_item *items, int n_items,
                                 const pmf_run_params *p, pmf_run **out);

/* Launch of a batched run (more than one item).  PMF_BATCH_PACKED (the
 * default for FP32 chain batches): one persistent launch per 1e5-step chunk
 * for the whole batch; each CTA (16 warps, one per SM) takes (segment, pack)
 * work items from a device queue, a pack being up to 16 / G replicas of one
 * item simulated side by side by teams of G warps (G = 2, 4, 8 or 16: the
 * smallest allowed team size whose 16 / G replicas fit the CTA's shared
 * memory, allowed being G >= 4 under packing policy `shift` = 0 (the
 * default), G >= 2 under 1 and G >= 8 under 2; chains too long for a full
 * CTA at any allowed size take the size that keeps the most warps busy,
 * 16 if it fits); packs are
 * queued costliest first, segment-major, and a pack's segment waits
 * (bounded, as for single runs) for its previous one.  Every replica then
 * runs the force schedule of G warps, so its trajectory is bit-identical to
 * a per-item launch with G warps per replica.  PMF_BATCH_GRAPH: the
 * per-item launches of pmf_run_batch_prepare's graph (FP64 batches always).
 * PMF_EINVAL for a packed launch of an FP64 chain, a chain too long to fit,
 * or a non-window run; PMF_ESTATE while the run is in flight.
 * pmf_run_get_batch_launch reports the mode, shift, the number of packs and
 * CTAs (0 in graph mode) and the team size of each item (teams[capacity],
 * may be NULL; 0 in graph mode).
 * pmf_run_batch_autotune times probe_steps steps of the whole batch (a
 * warm-up and the best of two launches) in graph mode and in packed mode for
 * every policy that gives different team sizes, and keeps the fastest; the
 * probes overwrite the run's samples, so call it before the real launch.
 * The paper runs one path at a time; packing many is this library's. */
enum { PMF_BATCH_GRAPH = 0, PMF_BATCH_PACKED = 1 };
pmf_status pmf_run_set_batch_launch(pmf_run *run, int mode, int shift);
pmf_status pmf_run_get_batch_launch(pmf_run *run, int *mode, int *shift, int *packs, int *ctas, int *teams,
                                    int capacity);
pmf_status pmf_run_batch_autotune(pmf_run *run, int64_t probe_steps, double *best_ms);

/* Constant-velocity pulling, the steered-MD comparator the paper measures
 * against (Sec. I, the work -v k int (x - lambda_1 - v t) dt): p->replicas
 * simulations start from x_o with the trap at lambda1, relax p->n_equil
 * steps (n_equil < 0: 10 % of n_steps), then the trap centre advances by
 * velocity * dt per step for the remaining steps; each move from lambda to
 * lambda' does the work of Eq. (9), k/2 (lambda' - lambda)(lambda' + lambda -
 * 2 x), at the reaction coordinate of that moment (chain: at the force
 * evaluation ending a step; 1D: before the step).  Every sample_stride steps
 * of pulling, x (pmf_x_samples, one window) and the accumulated work
 * (pmf_smd_work, FP64, [replica][record]) are recorded; record j is at trap
 * position lambda1 + velocity dt (j + 1) sample_stride.  pmf_smd_free_energy
 * gives per record: dF_JE = -kT ln <exp(-W/kT)> over the replicas (Eq. (1)),
 * dF_cumulant = <W> - var(W)/2kT (the second-order cumulant estimate of the
 * PMF method), <W>, var(W) (divisor replicas) and <x>; arrays of capacity
 * >= the record count, any may be NULL. */
pmf_status pmf_run_prepare_smd(pmf_system *sys, double lambda1, double velocity, const pmf_run_params *p,
                               pmf_run **out);
pmf_status pmf_smd_work(const pmf_run *run, double *out, size_t capacity, size_t *n_written);
pmf_status pmf_smd_free_energy(const pmf_run *run, double *lambda, double *dF_JE, double *dF_cumulant,
                               double *W_mean, double *W_var, double *mean_x, int capacity);

/* Shape of a run's sample store: x[w][r][t], t fastest; window w holds
 * replicas * samples_per_window[w] floats starting at sample_offset[w]. */
typedef struct {
    int n_windows;
    int replicas;
    int64_t total_samples;
    int64_t samples_per_window[PMF_MAX_RUN_WINDOWS];
    int64_t sample_offset[PMF_MAX_RUN_WINDOWS];
} pmf_run_info;
pmf_status pmf_get_run_info(const pmf_run *run, pmf_run_info *info);

/* Copy the recorded x samples (FP32, layout of pmf_run_info) to the host
 * buffer out[capacity].  If capacity is too small: PMF_EINVAL and
 * *n_written = the required count. */
pmf_status pmf_x_samples(const pmf_run *run, float *out, size_t capacity, size_t *n_written);

enum { PMF_WORK_PER_WINDOW_INCREMENT = 0, PMF_WORK_PAIRED_CUMULATIVE = 1 };
/* Work samples of Eq. (9), FP64, computed on the GPU:
 *   PER_WINDOW_INCREMENT: w_i = k/2 (lambda_{i+1} - lambda_i)(lambda_{i+1} + lambda_i - 2 x_i)
 *     for windows i = 0..s-2, layout [i][r][t] (the sample layout without
 *     the last window);
 *   PAIRED_CUMULATIVE: W_j(r, t) = sum_{i < j} w_i(x_i[r][t]), the work of
 *     the force-versus-extension curve formed by replica r, sample t in every
 *     window, layout [j = 1..s-1][r][t]; needs equal samples per window.
 * Capacity handling as for pmf_x_samples. */
pmf_status pmf_work_samples(const pmf_run *run, int mode, double *out, size_t capacity,
                            size_t *n_written);

/*
 * Free-energy estimates (all energies in the system's energy unit), per
 * profile point j = 0..s-1 (value at lambda_1 is 0), computed on the GPU in
 * FP64 from the x samples:
 *   dF_JE       Eq. (12): sum_{i<j} -kT ln <exp(-w_i/kT)>_i  (the average over
 *               all combinations of samples factorises over the independent
 *               windows; max-shifted log-sum-exp with compensated sums)
 *   dF_fluct    Eq. (14): sum_{i<j} k D_i (lambda_i - <x_i>), D_i = lambda_{i+1} - lambda_i
 *   dF_G        Eq. (13): sum_{i<j} [k D_i^2/2 (1 - gamma_i^2) + k D_i (lambda_i - <x_i>)]
 *   dF_com      (dF_JE + dF_fluct)/2, uncertainty (dF_JE - dF_fluct)/2 (Sec. V)
 *   se_JE, se_fluct  delete-one-replica jackknife, variances summed over windows
 *   var_ZW      sigma_W^2/Q + sigma_W^4/(2 kT^2 (Q-1)) (Sec. IV A), Q = min_i n_i
 *   W_mean      <W_mech> = sum_{i<j} <w_i> (Fig. 3b)
 *   acc_force   dF_fluct / (lambda_j - lambda_1), 0 at j = 0 (Fig. 4b)
 * per window i: mean_x, var_x (divisor n), gamma2 = k var_x / kT (Eq. (13)).
 * Any array pointer may be NULL; each non-NULL array holds >= n_windows.
 */
typedef struct {
    int capacity;               /* length of every non-NULL array               */
    double *lambda, *dF_JE, *dF_fluct, *dF_G, *dF_com, *uncertainty;
    double *se_JE, *se_fluct, *var_ZW, *W_mean, *acc_force;
    double *mean_x, *var_x, *gamma2;
} pmf_free_energy_result;

pmf_status pmf_free_energy(const pmf_run *run, pmf_free_energy_result *res);

/* The estimates above for item `item` of a batched run (its own windows
 * only, profile value 0 at its first window); res->capacity >= the item's
 * n_windows >= 2.  Works on single-item runs too (item 0).  Synchronous. */
pmf_status pmf_free_energy_item(const pmf_run *run, int item, pmf_free_energy_result *res);

/* Enqueue the FP64 reductions behind pmf_free_energy on the library stream
 * and return at once; the results stay in device memory until the next
 * pmf_free_energy call copies them (without recomputing).  Needs a launched
 * run (PMF_ESTATE otherwise). */
pmf_status pmf_run_reduce(pmf_run *run);

/* The exchange step of a run sharded over processes or GPUs (each shard
 * runs every window with its own replicas, disjoint uids).  pmf_run_partials
 * computes the run's per-replica partial sums on the GPU and copies them to
 * out[capacity] (host), FP64, [window][replica][5] =
 *   {m = min_t w_i, S = sum_t exp(-(w_i - m)/kT), n, sum_t (x - lambda_i),
 *    sum_t (x - lambda_i)^2}
 * with w_i of Eq. (9) (w = 0 in the last window).  Single-item runs; capacity
 * handling as for pmf_x_samples.  Shards' partials are merged by
 * concatenating them along the replica axis of every window (the max-shifted
 * sums S are rescaled to a common shift inside the combination), and
 * pmf_free_energy_from_partials turns partials[n_windows][replicas][5]
 * (host) into every estimate of pmf_free_energy, identical to a single run
 * over the union of the replicas up to the order of the sums. */
pmf_status pmf_run_partials(const pmf_run *run, double *out, size_t capacity, size_t *n_written);
pmf_status pmf_free_energy_from_partials(const double *partials, const double *lambda, int n_windows,
                                         int replicas, double k, double kT, pmf_free_energy_result *res);

/* Work distributions of App. C.  Each window's x samples are counted into
 * n_x bins [x_lo + j dx, x_lo + (j + 1) dx) (rho_i, divided by the window's
 * sample count; samples outside are lost).  The distribution of the work
 * accumulated over the first i - 1 pulling steps, Omega_i, lives on the bins
 * W = b dw, b = -M..M; Omega_1 is all at W = 0 and Omega_{i+1} adds the
 * increment of Eq. (9) at every x bin of window i, weighted by rho_i.  With
 * left_edge = 0 (the default reading) a bin stands for its centre and a work
 * value goes to the nearest bin; left_edge = 1 follows the rule as printed
 * (left edges, floor, and the W = 0 bin smoothed as the mean of its
 * neighbours after every step).  The recursion runs through Omega_s.
 * Outputs (each may be NULL): omega[s][2M + 1] (host, capacity in doubles),
 * dF_JE[i] = -kT ln sum_b Omega_i(b) exp(-b dw / kT) / sum_b Omega_i(b),
 * var_ZW[i] = the App. C variance with sigma_W of Omega_i and Q its non-zero
 * bins, lost[i] = 1 - sum_b Omega_i(b): probability that left the W or x
 * range (with left_edge = 1 also the change the smoothing makes).  The run must
 * be finished and single-item; every window needs a sample inside the x
 * range.  As dx, dw -> 0 (bin centres) dF_JE tends to pmf_free_energy's. */
typedef struct {
    double x_lo, dx;            /* x bins                                        */
    int n_x;                    /* number of x bins (<= 2^26)                    */
    double dw;                  /* work bin width                                */
    int M;                      /* work bins b = -M..M (<= 2^24)                 */
    int left_edge;              /* 0: bin centres, nearest bin; 1: as printed    */
} pmf_hist_params;
pmf_status pmf_work_distributions(const pmf_run *run, const pmf_hist_params *hp, double *omega,
                                  size_t omega_capacity, double *dF_JE, double *var_ZW, double *lost);

/* State free energy of Eq. (15): G(lambda_j, lambda_1) = dF^JE(lambda_j,
 * lambda_1, k) - dF(lambda_1, k) at every profile point j (so the value at
 * lambda_1 is -dF(lambda_1, k)), where dF(lambda_1, k) = F(lambda_1, k) - F_0
 * is the free energy of turning the trap on, from Eq. (5):
 * kT ln <exp(k/2 (x_1 - lambda_1)^2 / kT)> over the first window's samples
 * (max-shifted log-sum-exp, compensated sums, FP64 on the GPU).  se_G: the
 * delete-one-replica jackknife (the first window's replica r is left out of
 * its JE increment and of the turn-on average together; the other windows'
 * JE variances are added).  G and se_G (host) hold >= n_windows values (may
 * be NULL), *dF_turn_on (host, may be NULL) receives dF(lambda_1, k).  Eq. (5)
 * converges only when the trapped first window samples the whole support of
 * the unbiased ensemble (a soft trap); with a stiff trap the turn-on term is
 * biased low.  The run must be finished and a single-path window run
 * (PMF_EINVAL for batches and pulled runs); capacity >= n_windows. */
pmf_status pmf_state_free_energy(pmf_run *run, double *G, double *se_G, double *dF_turn_on, int capacity);
/* The same on caller-supplied samples (arguments as for
 * pmf_free_energy_from_samples; 1 <= n_windows <= 1024). */
pmf_status pmf_state_free_energy_from_samples(const float *x, int x_on_device, const double *lambda, int n_windows,
                                              int replicas, const int64_t *samples_per_window, double k, double kT,
                                              double *G, double *se_G, double *dF_turn_on);

/* The same reduction on caller-supplied samples x (layout of pmf_run_info
 * with `replicas` and samples_per_window[n_windows]); x is a host pointer
 * (x_on_device = 0) or a device pointer (x_on_device = 1). */
pmf_status pmf_free_energy_from_samples(const float *x, int x_on_device, const double *lambda,
                                        int n_windows, int replicas,
                                        const int64_t *samples_per_window, double k, double kT,
                                        pmf_free_energy_result *res);

/* Allocation-free form of pmf_free_energy_from_samples, for callers that
 * must not allocate GPU memory: for instance a host application whose own
 * pool has already reserved the device memory, or a latency-critical loop
 * that cannot afford the device-wide synchronisation of cudaMalloc/cudaFree.
 * The paper has no counterpart; it is a library-interface convenience.
 *   x       device pointer, FP32 samples [n_windows][replicas][samples_per_window]
 *   lambda  device pointer, n_windows window centres (strictly monotone)
 *   out     device pointer, 14 * n_windows doubles: the arrays of
 *           pmf_free_energy_result in its field order (lambda, dF_JE, dF_fluct,
 *           dF_G, dF_com, uncertainty, se_JE, se_fluct, var_ZW, W_mean,
 *           acc_force, mean_x, var_x, gamma2), each n_windows long
 * Limits: 2 <= n_windows <= 1024, n_windows * replicas <= 65536,
 * samples_per_window >= 1; larger sizes return PMF_EINVAL.
 * The call only enqueues kernels on the library stream and returns; the
 * results are valid once that stream has reached this point.  Its scratch is
 * a fixed array (about 2.7 MB) that every GPU which loads the library keeps
 * until the process exits, shared by all calls on that GPU: calls whose work
 * overlaps on the GPU race and must be serialised by the caller.  The first
 * call on a device looks up that array's device address (with the device
 * current); make that first call before any stream capture begins.  No call
 * allocates or frees memory. */
pmf_status pmf_free_energy_noalloc(const float *x, const double *lambda, int n_windows, int replicas,
                                   int64_t samples_per_window, double k, double kT, double *out);

/* Final state of every replica: pos/vel [window][replica][bead][3] (chain) or
 * [window][replica] (1D, vel unused); sequential runs: [replica][bead][3] or
 * [replica].  Capacity in doubles of each buffer. */
pmf_status pmf_final_state(const pmf_run *run, double *pos, double *vel, size_t capacity,
                           size_t *n_written);

/* ---- batching / autotuning ----------------------------------------------
 * Warps per replica CTA of chain `chain` (4, 5, 6 or 8 for FP32; FP64 uses 4);
 * the host schedule of the nonbonded phase is rebuilt for the new count.
 * Results are bit-reproducible for a given count; different counts sum the
 * forces in different orders. */
pmf_status pmf_chain_set_warps(pmf_system *sys, int chain, int warps);
/* Launch shape of chain `chain` in single-item runs.  ctas < 0: one CTA per
 * replica, every replica's steps in one launch per 1e5-step chunk.
 * ctas >= 0: persistent launch of min(ctas, replicas) CTAs (ctas = 0: every
 * CTA slot the GPU holds at once) that take work items of seg_steps steps
 * (0: 1000) of one replica from a device queue, in segment-major order
 * (ctas = 0 picks: every slot if the replicas fill them, else a whole number
 * of CTAs per SM when that is at least 3, else one CTA per replica); a
 * replica's next segment waits (at most 60 s, then PMF_ETIMEOUT) until its
 * previous one has stored the state.  Replicas thus migrate between CTAs and
 * no SM idles when the replica count is not a multiple of the SM count.
 * Trajectories are bit-identical for every shape (the state record holds
 * the whole integrator state between segments).  Default: ctas = 0,
 * seg_steps = 1000.  Batched runs always use one CTA per replica. */
pmf_status pmf_chain_set_grid(pmf_system *sys, int chain, int ctas, int seg_steps);
/* Schedule cost model of chain `chain` (see pmf_chain_schedule_variant; the
 * work schedule is rebuilt, results are bit-reproducible for a given
 * variant and warp count).  PMF_EINVAL for a variant out of range. */
pmf_status pmf_chain_set_schedule(pmf_system *sys, int chain, int variant);
pmf_status pmf_chain_get_schedule(const pmf_system *sys, int chain, int *variant);
/* The current warps per replica, ctas and seg_steps of chain `chain` (as set
 * by the calls above or chosen by pmf_chain_autotune); NULL outputs skipped. */
pmf_status pmf_chain_get_launch(const pmf_system *sys, int chain, int *warps, int *ctas, int *seg_steps);
/* Time probe_steps steps of the given run (every window and replica, one
 * warm-up launch and the best of two timed launches each; use several
 * thousand steps so the persistent segments dominate the launch tail) for
 * each warp count and each of two persistent
 * launch shapes (ctas = 0 and ctas = one per replica, see
 * pmf_chain_set_grid), keep the fastest, then, for FP32, time each schedule
 * cost model that gives a different schedule for that shape and keep the
 * fastest; *best_warps and *best_ms (may be NULL) report the warp count
 * chosen and its probe time. */
pmf_status pmf_chain_autotune(pmf_system *sys, const double *lambda, int n_windows, const pmf_run_params *p,
                              int probe_steps, int *best_warps, double *best_ms);

/* ---- learned window placement: surrogate MLP ---------------------------
 * A small network lambda -> (mu, log sigma^2) of the reaction coordinate,
 * 1 -> 64 -> 64 -> 2 with SiLU, trained on a run's (lambda_i, x) samples by
 * the Gaussian negative log-likelihood 0.5 [log sigma^2 + (x - mu)^2 / sigma^2]
 * with Adam.  It models the Gaussian rho(x_i) of Sec. II (the text before
 * Eq. (13)) as a smooth function of lambda, so the overlap of adjacent x
 * distributions (the criterion of Sec. III, Sec. IV B and Sec. V (iii)) can be
 * predicted between windows.  Inputs and targets are normalised as
 * lambda' = (lambda - c) / h, x' = (x - c) / h.  The 64 x 64 layer runs on
 * the tensor cores in BF16 with FP32 accumulation (forward and backward);
 * FP32 master weights.  Parameters are packed as W1[64], b1[64],
 * W2[64][64] (row = output), b2[64], W3[2][64], b3[2]. */
#define PMF_MLP_PARAMS 4418
typedef struct pmf_mlp pmf_mlp;
/* params: PMF_MLP_PARAMS initial FP32 weights (host, copied). */
pmf_status pmf_mlp_create(const float *params, double c, double h, pmf_mlp **out);
void pmf_mlp_destroy(pmf_mlp *mlp);
/* Current FP32 weights into params[PMF_MLP_PARAMS] (host). */
pmf_status pmf_mlp_get_params(const pmf_mlp *mlp, float *params);
/* mu[n], log_var[n] (host) at lambda[n] (host), physical units. */
pmf_status pmf_mlp_predict(pmf_mlp *mlp, const double *lambda, int n, double *mu, double *log_var);
/* Gradient grad[PMF_MLP_PARAMS] (host) of the mean normalised NLL over the
 * samples (lambda[n], x[n]) (host) and that loss (*loss, may be NULL);
 * weights unchanged. */
pmf_status pmf_mlp_gradient(pmf_mlp *mlp, const double *lambda, const float *x, int n, float *grad, double *loss);
/* Adam training on a finished run: `steps` updates, each on `batch` samples
 * (rounded up to a multiple of 128) drawn uniformly from the run's sample
 * store by Philox4x32-10 with key seed, counter (j, step, 0, 3), index =
 * (word1 << 32 | word0) mod total; the sample's window gives lambda.  lr is
 * the Adam step size (beta 0.9 / 0.999, eps 1e-8).  *loss (may be NULL)
 * receives the last batch's mean normalised NLL.  PMF_ETIMEOUT if a tensor
 * core completion wait ran out (the kernel then stops and frees its tensor
 * memory). */
pmf_status pmf_mlp_train(pmf_mlp *mlp, const pmf_run *run, int steps, int batch, double lr, uint64_t seed,
                         double *loss);
/* How training (pmf_mlp_train and the adaptive protocol's rounds) runs on
 * the GPU.  split = 1 (the default): every Adam step is one launch with a
 * CTA per 128-sample tile of the batch, each writing its tile's gradient,
 * then an update launch that sums the tiles in tile order and applies Adam;
 * the scratch ([tiles][PMF_MLP_PARAMS] floats) is allocated on first use and
 * kept with the surrogate.  split = 0: one CTA runs all steps, the tiles of
 * a step one after another.  Both draw the same mini-batches; they differ
 * only in FP32 summation order.  PMF_EINVAL for other values. */
pmf_status pmf_mlp_set_split(pmf_mlp *mlp, int split);

/* ---- adaptive protocol: surrogate-guided window insertion -----------------
 * Starting from windows lambda0[n0] (a coarse PPP run from x_o), repeat up
 * to max_rounds times: train the surrogate on the samples of every window
 * so far, predict N(mu, sigma^2) of x at each window, and insert the midpoint
 * of every adjacent pair whose predicted overlap coefficient
 * int min(p_i, p_{i+1}) is below overlap_threshold (the paper's criterion
 * that adjacent distributions of x overlap comparably to their spread,
 * Sec. III, Sec. IV B, Sec. V (iii)).  Each inserted window's replicas start
 * from the stored end states of its two neighbours whose final x is nearest
 * the predicted mean (replica r takes the candidate of rank r mod count) and
 * run with the same parameters and fresh replica uids (with
 * continue_windows, every current window continues in the same launch).
 * The estimators of pmf_free_energy are then evaluated on the merged
 * non-uniform grid.
 * gpu_seconds sums the device time of the simulations, the training, the
 * predictions, the seeding and the reductions (CUDA events on the library
 * stream).  Unless the caller set the chain's warp count
 * (pmf_chain_set_warps or pmf_chain_autotune), each FP32 chain launch of the
 * protocol uses 8 warps per replica when it has fewer than three replicas
 * per SM and 4 otherwise; the chain is back at 4 on return. */
/* Optional record of the protocol's decisions (caller-owned host arrays;
 * a NULL array is not filled).  Round q (q < max_rounds) stores, for the
 * n_windows[q] windows it started from (path order):
 *   lambda, mu, log_var  [q][max_windows]: centres and the surrogate's
 *                        prediction there;
 *   ovl                  [q][max_windows]: OVL of windows i and i + 1;
 * and for the n_inserted[q] windows it inserted (path order):
 *   inserted, target     [q][max_windows]: centres and the predicted mean x
 *                        there (the seeding target);
 *   cand_x               [q][max_windows][2 replicas]: final x of each seeding
 *                        candidate (c < replicas: replica c of the left
 *                        neighbour, else replica c - replicas of the right);
 *   seed                 [q][max_windows][replicas]: the candidate each replica
 *                        of the inserted window started from.
 * With train_on_gap, data_ovl [q][max_windows] holds the OVL of windows i
 * and i + 1 from the measured moments of their samples, and trained[q] is 1
 * if round q trained the surrogate (a gap was found), else 0 (the round
 * stopped the protocol; its mu, log_var and ovl are NaN).  Without it
 * trained[q] is 1 and data_ovl is not written.
 * rounds receives the number of rounds recorded (the last one may insert
 * nothing).  max_windows must be >= pmf_adaptive_params.max_windows and
 * replicas = pmf_run_params.replicas (<= 2048), else PMF_EINVAL. */
typedef struct {
    int max_rounds, max_windows, replicas;
    int rounds;
    int *n_windows, *n_inserted;
    double *lambda, *mu, *log_var, *ovl;
    double *inserted, *target, *cand_x;
    int *seed;
    double *data_ovl;
    int *trained;
} pmf_adaptive_trace;

typedef struct {
    double overlap_threshold;   /* e.g. 0.3                                   */
    int max_rounds;             /* insertion rounds (>= 0)                    */
    int max_windows;            /* cap on the total window count (<= 1024)    */
    int mlp_steps, mlp_batch;   /* Adam updates and batch per round           */
    double mlp_lr;
    uint64_t mlp_seed;
    const float *mlp_init;      /* PMF_MLP_PARAMS initial weights (host)      */
    pmf_adaptive_trace *trace;  /* optional decision record (NULL: none)      */
    int continue_windows;       /* 1: every round runs all windows in one launch:
                                   the current ones continue for another n_steps
                                   from their own replicas' end states (replica
                                   r from replica r; fresh uids and velocities),
                                   the inserted ones start seeded; the estimate
                                   uses each window's latest run.  0: later
                                   rounds run the inserted windows only        */
    int train_on_gap;           /* 1: a round first measures the Gaussian
                                   moments (mean, population variance) of every
                                   window's samples and the OVL of each
                                   adjacent pair; if none is below
                                   overlap_threshold the protocol stops there
                                   without training (no window would need a
                                   neighbour).  0: every round trains.         */
} pmf_adaptive_params;

typedef struct {
    int n_windows;              /* final window count                         */
    int rounds;                 /* rounds that inserted windows               */
    int inserted;               /* windows inserted in total                  */
    double gpu_seconds;
    double mlp_loss;            /* last training batch loss                    */
    double lambda[1024];        /* final window centres, in path order        */
} pmf_adaptive_info;

/* res arrays must hold at least max_windows entries (res->capacity). */
pmf_status pmf_run_adaptive(pmf_system *sys, const double *lambda0, int n0, const pmf_run_params *p,
                            const pmf_adaptive_params *ap, pmf_adaptive_info *info, pmf_free_energy_result *res);

/* ---- kernel-level entry points used by the parity tests ---------------- */

/* Test hook of the bounded device wait (no counterpart in the paper): the
 * next launches of this single-item chain run start their persistent work
 * queue at item first_item (items are segment-major, item = segment x
 * (n_windows x replicas) + replica) instead of 0; the items before it never
 * run.  With first_item = n_windows x replicas every replica's second
 * segment waits for a first segment that never ran, so the launch ends by
 * itself after segment_wait_s with PMF_ETIMEOUT from pmf_run_wait.  0
 * restores the normal run.  PMF_EINVAL for other run kinds, PMF_ESTATE while
 * the run is in flight. */
pmf_status pmf_run_set_queue_start(pmf_run *run, int64_t first_item);

/* The integrator's Philox4x32-10 and Box-Muller on the GPU: blocks with
 * counters (c0 + i, c1, c2, c3), key (seed lo, seed hi), i < n_blocks.
 * raw[4 n_blocks] uint32 and normals[4 n_blocks] (FP32 as used by the FP32
 * integrator) are host buffers; either may be NULL. */
pmf_status pmf_philox(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                      int n_blocks, uint32_t *raw, float *normals);

/* Forces -grad H(lambda, x) of chain `chain` at positions pos[N][3] (host),
 * evaluated by the integrator's own force phase in the system's precision;
 * forces[N][3] host output. */
pmf_status pmf_chain_forces(pmf_system *sys, int chain, const double *pos, double lambda,
                            double k, double *forces);

/* Overlap coefficients ovl[i] = int min(p_i, p_{i+1}) dx, i < n - 1, of the
 * Gaussians N(mu_i, exp(log_var_i)) (host arrays), computed by the kernel
 * the adaptive protocol uses. */
pmf_status pmf_overlap(const double *mu, const double *log_var, int n, double *ovl);

/* Host-side schedule of the nonbonded phase for a chain of N beads, NW
 * warps per CTA and the integration precision (no GPU needed): the ring
 * pieces each warp executes, as records of 7 ints (warp, I1, I2 or -1, J,
 * kind, near1, near2) in out[capacity]; *n_written receives the record
 * count.  A piece pairs the 32-bead i-tile I1 (and I2) with j-tile J; at
 * ring step t lane l meets j = J*32 + ((l mod W) + t) mod W:
 *   scalar (FP64):  0..3  W 32, t = 8k..8k+7        4, 5  W 32 diagonal, t = 1..8, 9..16
 *                   6, 7  W 16, t = 0..7, 8..15      8     W 16 diagonal, t = 1..8
 *                   9     W 8,  t = 0..7             10    W 8 diagonal, t = 1..4
 *   quad (FP32): lane l holds i-beads at ring indices l and l + 1 and meets
 *   ring positions l + t and l + t + D (D = 8 for W 32 and 16, 4 for W 8),
 *   t stepping by 2 (kinds 8 and 10 as above):
 *                   21    W 32, t = 1, 3, 5, 7       22    W 32, t = 17, 19, 21, 23
 *                   23    W 32 diagonal, t = 2, 4, 6, 8
 *                   24    W 16, t = 1, 3, 5, 7       25    W 8, t = 1, 3
 * near1/near2 flag i-tiles adjacent to J (exclusions |i - j| <= 2 possible).
 * Tiles are 32 beads except a last tile of 8, 16 or 32 (*padded receives the
 * padded bead count).  PMF_EINVAL if capacity < 7 * records. */
pmf_status pmf_chain_schedule(int N, int NW, int precision, int *out, size_t capacity, size_t *n_written,
                              int *padded);
/* The same for cost model `variant` of the FP32 schedule (0 ..
 * pmf_chain_schedule_variants() - 1; pmf_chain_schedule is variant 0).  The
 * FP32 pieces are dealt longest-first to the least loaded warp under an
 * estimated cost per ring step, per piece, per bonded pass and per noise
 * pass; the variants weight these differently (the bonded and noise passes
 * are latency-bound, so their true cost depends on the chain and the warp
 * count).  FP64 schedules do not depend on the variant. */
int pmf_chain_schedule_variants(void);
pmf_status pmf_chain_schedule_variant(int N, int NW, int precision, int variant, int *out, size_t capacity,
                                      size_t *n_written, int *padded);

/* Measured FP32 throughput of this GPU, the peak of the integrator's
 * roofline (its nonbonded loop is bound by the FP32 FMA pipe): every SM
 * runs `ctas_per_sm` CTAs of 512 threads (0: 4, i.e. full occupancy), each
 * thread `iters` iterations of eight independent FMA chains, scalar FFMA
 * (packed = 0) or packed f32x2 FFMA2 (packed = 1).  One warm-up launch, then
 * the best of `reps` timed launches (CUDA events on the library stream).
 * *tflops = flops / time (an FMA counts as two flops); *ms = that launch's
 * time.  iters >= 1, reps >= 1, else PMF_EINVAL; the probe allocates
 * 2 KB per CTA of device memory for its results. */
pmf_status pmf_fp32_peak(int packed, int ctas_per_sm, int iters, int reps, double *tflops, double *ms);

/* Measured FP64 FMA throughput (DFMA, same probe shape as pmf_fp32_peak,
 * 4 KB per CTA of device memory): the ceiling of the FP64 reductions, whose
 * one exp per sample makes them FP64-bound rather than HBM-bound on a GPU
 * with GB300's FP64 rate. */
pmf_status pmf_fp64_peak(int ctas_per_sm, int iters, int reps, double *tflops, double *ms);

/* Library stream: cudaStream_t passed as void* (NULL = legacy default). */
pmf_status pmf_set_stream(void *stream);

/* Thread-local description of the last failure ("" if none). */
const char *pmf_last_error(void);

/* Library version string. */
const char *pmf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PMF_H */
