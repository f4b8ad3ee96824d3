// Internal host-side interfaces of libpmf (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace pmf {

// Host copy of one chain (FP64, as given by the caller).
struct ChainHost {
    int N = 0;
    std::vector<double> sigma, epsilon, charge, mass, dih_k, dih_phase, pos0;
    double bond_k = 0, bond_r0 = 0, angle_k = 0, angle_theta0 = 0, coulomb_k = 0;
    int nonbonded = 1;
};

constexpr int kMaxRunWindows = 4096;
// Longest wait of a persistent chain launch for a replica's previous segment
// unless the run sets its own (a segment normally takes milliseconds).
constexpr unsigned long long kDefaultSegmentWaitNs = 60ull * 1000000000ull;
constexpr int kMaxBranches = 64;  // concurrent item branches of a batched run's graph

// Tiling of N beads into 32-bead tiles; the last tile has width 8, 16 or 32.
struct ChainGeometry {
    int N = 0, Np = 0, n_tiles = 0, w_last = 32;
};

// One ring piece of the nonbonded phase: i-tile I1 (and I2 >= 0 for a dual
// piece, -1 otherwise) against j-tile J with piece kind `kind` (ring width,
// first ring step, step count, diagonal; see piece_kind in chain.cu).
// near1 / near2: that i-tile neighbours J, so exclusions |i - j| <= 2 occur.
struct UnitDesc {
    int I1, I2, J, kind, near1, near2;
};

ChainGeometry chain_geometry(int N);
// FP32 FMA throughput probe (peak.cu): ctas CTAs of fp32_peak_threads()
// threads, one float per thread into out; *flops of the launch
cudaError_t fp32_peak_launch(bool packed, int ctas, int iters, float *out, double *flops, cudaStream_t st);
cudaError_t fp64_peak_launch(int ctas, int iters, double *out, double *flops, cudaStream_t st);
int fp32_peak_threads();
// packed: the FP32 quad pieces (kinds 8, 10, 21..26); else the scalar pieces
// (0..10); variant: the cost model of the FP32 assignment (0 .. kSchedVariants-1)
constexpr int kSchedVariants = 6;
std::vector<std::vector<UnitDesc>> chain_schedule(int N, int NW, bool packed, int variant = 0);

// Everything one launch of a simulation kernel needs about the run.
struct RunLaunch {
    void *state = nullptr;         // per-replica state (layout owned by the model)
    float *xout = nullptr;         // x samples
    const double *lambda = nullptr;
    const long long *nsteps_w = nullptr, *nequil_w = nullptr, *off_w = nullptr, *tw = nullptr;
    int *err = nullptr;
    double *force_out = nullptr;
    const double *start = nullptr;  // optional per-replica start state (chain [rep][N][3], 1D [rep])
    // persistent chain launches (single-item runs): work queue counter and
    // per-replica segment counters, both zeroed by the launch itself
    unsigned long long *queue = nullptr;
    int *done = nullptr;
    long long queue_start = 0;         // first item taken (> 0 only to test the bounded wait)
    unsigned long long wait_ns = 0;    // longest wait for a previous segment (0: kDefaultSegmentWaitNs)
    const volatile int *abort = nullptr;  // host-mapped stop flag, polled between items
    // sequential protocol: n_blocks simulations each visit every window for
    // window_steps steps (steps [0, n_windows x window_steps)); persistent only
    bool sequential = false;
    long long window_steps = 0;
    // constant-velocity pulling (one window): the trap advances smd_vdt per
    // step after the equilibration; accumulated work recorded into wout
    double smd_vdt = 0;
    double *wout = nullptr;
    // 1D model: buffer for the per-step noise-and-trap terms q_n of noise_steps
    // steps of every simulation
    double *noise = nullptr;
    long long noise_steps = 0;
    long long step_begin = 0, step_end = 0;
    int replicas = 0, stride = 1, n_blocks = 0;
    uint32_t uid_base = 0;
    unsigned long long seed = 0;
    double k = 0, kT = 1, dt = 0, gamma = 1;
};

struct PackPlan;
class ChainModel {
public:
    struct Impl;
    ChainModel();
    ~ChainModel();
    cudaError_t init(const ChainHost &h, int precision);
    cudaError_t launch(const RunLaunch &L, cudaStream_t st);
    int n_beads() const;
    int n_padded() const;
    int precision() const;
    size_t state_bytes_per_replica() const;
    size_t smem_bytes() const;
    int warps() const;
    cudaError_t set_warps(int NW);  // 4, 5, 6 or 8 warps per replica (FP64: 4)
    // cost model of the FP32 schedule (0 .. kSchedVariants-1); rebuilds it
    cudaError_t set_schedule_variant(int v);
    int schedule_variant() const;
    // Incremented by every set_warps (which reallocates the work schedule a
    // captured launch points at): a captured graph older than this is stale.
    unsigned generation() const;
    // Launch shape: ctas > 0 persistent with that many CTAs, 0 persistent
    // with every CTA slot of the GPU, < 0 one CTA per replica; seg_steps =
    // steps per persistent work item (0: 1000).  Bumps the generation.
    cudaError_t set_grid(int ctas, int seg_steps);
    int grid_ctas() const;
    int seg_steps() const;
    // FP32 packed batch launch: the schedule of team size G (cached on the
    // device) and the shared memory of one replica team of that size
    cudaError_t team_schedule(int G, const int4 **units, const int **count, int *max_units);
    size_t team_slot_bytes(int G) const;

private:
    Impl *p;
    friend cudaError_t pack_plan_create(const std::vector<struct PackItemSpec> &, const std::vector<int> &, int,
                                        PackPlan **);
};

// Packed persistent launch of a batch (chain.cu): one CTA of 16 warps per
// SM runs packs of 16 / G replicas of one item, G warps each (teams), from a
// device queue of (segment, pack) items.  L: the item's one-CTA-per-replica
// launch fields (state, sample layout, lambda, uid base, n_blocks =
// replicas of the item).
struct PackItemSpec {
    ChainModel *model;
    RunLaunch L;
};
// team size of a chain under packing policy 0 (smallest G >= 4 whose 16 / G
// replicas fit a CTA), 1 (G >= 2) or 2 (G >= 8); -1: does not fit
int pack_team_choice(const ChainModel &m, int policy);
cudaError_t pack_plan_create(const std::vector<PackItemSpec> &items, const std::vector<int> &teams, int seg_steps,
                             PackPlan **out);
cudaError_t pack_plan_launch(PackPlan *plan, long long step_begin, long long step_end, cudaStream_t st);
void pack_plan_destroy(PackPlan *plan);
int pack_plan_packs(const PackPlan *plan);
int pack_plan_grid(const PackPlan *plan);
size_t pack_plan_smem(const PackPlan *plan);

struct Od1dParams {
    double a = 2.0, x0 = -1.0;
};
// Launches the noise pre-pass and the integration per block of noise_steps
// steps; the state holds x and the pulling work per simulation (2 doubles).
cudaError_t od1d_launch(const Od1dParams &m, const RunLaunch &L, int n_rep, cudaStream_t st);
long long od1d_noise_steps(int n_rep);

// FP64 reductions of x samples into the estimators.
struct ReduceLayout {
    const float *x = nullptr;          // device samples
    const double *lambda = nullptr;    // device [s]
    const long long *off_w = nullptr;  // device [s]
    const long long *tw = nullptr;     // device [s]
    int n_windows = 0, replicas = 0;
    double k = 0, kT = 1;
};
// Device output block: 14 arrays of n_windows doubles, in this order.
enum ResultField {
    kResLambda = 0, kResJE, kResFluct, kResG, kResCom, kResUnc, kResSeJE, kResSeFluct,
    kResVarZW, kResWMean, kResAccForce, kResMeanX, kResVarX, kResGamma2, kResFields
};
// scratch: device buffer of reduce_scratch_bytes(); out: device [kResFields][n_windows]
size_t reduce_scratch_bytes(int n_windows, int replicas);
cudaError_t reduce_launch(const ReduceLayout &L, void *scratch, double *out, cudaStream_t st);
// The two halves of reduce_launch.  Per-replica partials, 5 doubles each,
// [window][replica]: {min w, sum exp(-(w - min)/kT), n, sum (x - lambda_i),
// sum (x - lambda_i)^2}; combine turns them into the results (window_scratch:
// >= reduce_scratch_bytes - partial_bytes).
constexpr int kPartialDoubles = 5;
// Constant-velocity pulling estimators per record j of T: out[5][T] =
// {JE, mean - var / 2kT, mean work, work variance (divisor R), mean x}.
cudaError_t smd_stats_launch(const double *W, const float *x, int R, long long T, double kT, double *out,
                             cudaStream_t st);
size_t partial_bytes(int n_windows, int replicas);
cudaError_t partials_launch(const ReduceLayout &L, void *partials, cudaStream_t st);
cudaError_t combine_launch(const ReduceLayout &L, const void *partials, void *window_scratch, double *out,
                           cudaStream_t st);
// Allocation-free reduction: scratch in a fixed device array, equal samples
// per window, all pointers on the device.
constexpr int kNoAllocMaxWindows = 1024;
constexpr long long kNoAllocMaxWindowReplicas = 65536;  // n_windows * replicas
cudaError_t reduce_noalloc_launch(const float *x, const double *lambda, int n_windows, int replicas,
                                  long long samples_per_window, double k, double kT, double *out, cudaStream_t st);
// Eq. (5) / Eq. (15) after reduce_launch filled `scratch`: out[2 s + 1] =
// G(lambda_j, lambda_1) [s], its standard error [s], dF(lambda_1, k);
// turn_partials: device buffer of partial_bytes(1, replicas).
cudaError_t state_launch(const ReduceLayout &L, void *scratch, void *turn_partials, double *out, cudaStream_t st);
cudaError_t work_samples_launch(const ReduceLayout &L, int mode, long long samples_per_replica, double *out,
                                cudaStream_t st);

// Surrogate MLP (mlp.cu)
constexpr int kMlpParams = 64 + 64 + 64 * 64 + 64 + 2 * 64 + 2;
constexpr int kMlpTile = 128;  // samples per tcgen05 tile (one CTA's rows)
struct MlpLaunch {
    float *params = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    int adam_t = 0;
    double lr = 1e-3, c = 0, h = 1;
    const double *lam_in = nullptr;
    const float *x_in = nullptr;
    int n = 0;
    const float *xs = nullptr;
    const double *win_lambda = nullptr;
    const long long *win_off = nullptr, *win_tw = nullptr;
    int n_windows = 0, replicas = 0;
    long long total = 0;
    int mode = 0, steps = 0, batch = 0;
    unsigned long long seed = 0;
    double *out_mu = nullptr, *out_logvar = nullptr;
    float *out_grad = nullptr;
    double *out_loss = nullptr;
    int *err = nullptr;
    // training (mode 2) with split: one CTA per 128-sample tile and an
    // update kernel per step; tile_grad [tile_cap][kMlpParams] and
    // tile_loss [tile_cap] are the caller's scratch
    bool split = false;
    float *tile_grad = nullptr;
    double *tile_loss = nullptr;
    int tile_cap = 0;
};
cudaError_t mlp_launch(const MlpLaunch &L, cudaStream_t st);

// Learned window placement (adaptive.cu)
cudaError_t overlap_launch(const double *mu, const double *log_var, int n, double *ovl, cudaStream_t st);
// mu[w], log_var[w]: mean and log population variance of window w's samples
// x[off[w] .. off[w] + tw[w] * replicas) (a merged sample store)
cudaError_t moments_launch(const float *x, const long long *off, const long long *tw, int replicas, int n,
                           double *mu, double *log_var, cudaStream_t st);
constexpr int kMaxSeedCandidates = 4096;
struct SeedJob {
    double target;                         // predicted mean x at the inserted window
    int n_cand;                            // candidates (end states of the neighbours)
    const void *cand[kMaxSeedCandidates];  // positions (chain: 4 values per bead) or x (1D)
};
// choice (optional, [n_jobs][replicas]): candidate each replica took;
// cand_x (optional, [n_jobs][max_cand]): each candidate's final x
cudaError_t seed_launch(const SeedJob *jobs, int n_jobs, int max_cand, int N, int Np, int replicas, bool fp64,
                        double *start, int *choice, double *cand_x, cudaStream_t st);

// Work distributions of App. C (histogram.cu)
struct HistStep {
    double x_lo = 0, dx = 1, dw = 1;  // x bins and work bin width
    double hk = 0, d = 0, lsum = 0;   // k/2, lambda_{i+1} - lambda_i, lambda_{i+1} + lambda_i
    int left_edge = 0;                // the printed rule: bin left edges and floor
    long long jmin = 0, jmax = -1;    // occupied x bins of the window
    long long gmin = 0, gmax = -1;    // support of the shift distribution
};
cudaError_t hist_count_launch(const float *x, const long long *off_w, const long long *tw, int n_windows, int replicas,
                              double x_lo, double dx, int n_x, unsigned long long *cnt, unsigned long long *outside,
                              int *jmin, int *jmax, cudaStream_t st);
long long hist_shift_host(const HistStep &h, long long j);
cudaError_t hist_step_launch(const HistStep &h, const unsigned long long *cnt_w, double inv_n, double *g,
                             const double *in, long long in_lo, long long in_hi, double *out, long long out_lo,
                             long long out_hi, long long M, cudaStream_t st);
cudaError_t hist_stats_launch(const double *om, int n_windows, long long M, double dw, double kT, const long long *sup,
                              double *stats, cudaStream_t st);

cudaError_t philox_launch(unsigned long long seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int n,
                          uint32_t *raw, float *normals, cudaStream_t st);

}  // namespace pmf
