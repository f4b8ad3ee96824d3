// C ABI of libpmf: handles, argument checks, orchestration of the kernels.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "../../include/pmf.h"
#include "common.cuh"
#include "internal.h"

using namespace pmf;

namespace {

thread_local std::string g_err;
cudaStream_t g_stream = nullptr;

pmf_status fail(pmf_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}
pmf_status cuda_fail(cudaError_t e, const char *where)
{
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PMF_ENOMEM : PMF_ECUDA;
}
#define CK(call, where)                                          \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);      \
    } while (0)

pmf_status need_device()
{
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) return fail(PMF_ECUDA, "no CUDA device available (libpmf has no CPU path)");
    return PMF_OK;
}

// Device time of the work enqueued between start() and stop() on the
// library stream, accumulated over calls.
struct GpuTimer {
    double ms = 0.0;
    cudaEvent_t a = nullptr, b = nullptr;
    GpuTimer()
    {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~GpuTimer()
    {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
    void start() { cudaEventRecord(a, g_stream); }
    cudaError_t stop()
    {
        cudaEventRecord(b, g_stream);
        cudaError_t e = cudaEventSynchronize(b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
        ms += t;
        return e;
    }
};

template <typename T> cudaError_t upload(T **d, const T *h, size_t n)
{
    cudaError_t e = cudaMalloc(d, sizeof(T) * (n ? n : 1));
    if (e != cudaSuccess) return e;
    return n ? cudaMemcpy(*d, h, sizeof(T) * n, cudaMemcpyHostToDevice) : cudaSuccess;
}

}  // namespace

struct pmf_system {
    int model = 0, precision = 0;
    std::vector<std::unique_ptr<ChainModel>> chains;
    std::vector<char> warps_chosen;  // per chain: warps set by the caller or by autotuning
    Od1dParams od;
};

// One chain path of a run: windows [w0, w0 + nw) of the run use chain
// `chain`; their replica states start at byte state_off of d_state.
struct RunItem {
    int chain = 0, w0 = 0, nw = 0;
    size_t state_off = 0, state_stride = 0;
};

struct pmf_run {
    pmf_system *sys = nullptr;
    std::vector<RunItem> items;
    cudaStream_t cap = nullptr;        // private stream for graph capture
    std::vector<cudaStream_t> branch;  // capture-time fork streams (batch runs)
    std::vector<cudaEvent_t> fork_ev;  // [0]: fork point, [1 + b]: join of branch b
    cudaGraphExec_t graph = nullptr;   // captured launch sequence
    std::vector<unsigned> graph_gen;   // schedule generation per item at capture time
    int chain = 0, n_windows = 0, replicas = 0, stride = 1;
    bool sequential = false;  // sequential protocol: replicas visit the windows in order
    double smd_vdt = 0;       // constant-velocity pulling: trap advance per step
    double *d_w = nullptr;    // constant-velocity pulling: work at the records
    double *d_noise = nullptr;  // 1D model: q_n (noise and trap term) of a block of steps
    long long noise_steps = 0;
    double k = 0, kT = 1, dt = 0, gamma = 1, timeout_s = 0, segment_wait_s = 0;
    long long queue_start = 0;  // persistent chain launches: first work item (test hook)
    // batched FP32 chain runs: one packed persistent launch per chunk (mode 1)
    // or a graph of per-item launches (mode 0); team shift of the packing
    int batch_mode = 0, pack_shift = 0;
    PackPlan *pack = nullptr;
    long long probe_steps = 0;  // > 0: launches stop after this many steps (autotuning probes)
    int *h_abort = nullptr;     // host-mapped stop flag polled by the persistent chain launches
    int *d_abort = nullptr;     //   (its device alias)
    unsigned long long seed = 0;
    uint32_t uid_base = 0;
    std::vector<double> lambda;
    std::vector<long long> nsteps, nequil, off, tw;
    long long total = 0, max_steps = 0;
    double *d_lambda = nullptr;
    long long *d_nsteps = nullptr, *d_nequil = nullptr, *d_off = nullptr, *d_tw = nullptr;
    float *d_x = nullptr;
    void *d_state = nullptr;
    int *d_err = nullptr;
    void *d_scratch = nullptr;
    double *d_res = nullptr;
    double *d_start = nullptr;  // per-replica start state of a seeded run
    unsigned long long *d_queue = nullptr;  // persistent launch: work counter
    int *d_done = nullptr;                  // persistent launch: per-replica segments done
    cudaEvent_t done = nullptr;
    bool launched = false, finished = false, reduced = false;
    size_t state_bytes = 0;
    ~pmf_run()
    {
        if (launched && done) cudaEventSynchronize(done);  // kernels may still use the buffers
        cudaFree(d_lambda);
        cudaFree(d_nsteps);
        cudaFree(d_nequil);
        cudaFree(d_off);
        cudaFree(d_tw);
        cudaFree(d_x);
        cudaFree(d_state);
        cudaFree(d_err);
        cudaFree(d_scratch);
        cudaFree(d_res);
        cudaFree(d_start);
        cudaFree(d_queue);
        cudaFree(d_done);
        cudaFree(d_w);
        cudaFree(d_noise);
        if (h_abort) cudaFreeHost(h_abort);
        pack_plan_destroy(pack);
        if (done) cudaEventDestroy(done);
        if (graph) cudaGraphExecDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
        for (cudaStream_t b : branch) cudaStreamDestroy(b);
        for (cudaEvent_t e : fork_ev) cudaEventDestroy(e);
    }
};

static pmf_status need_finished(const pmf_run *run)
{
    if (!run) return fail(PMF_EINVAL, "null run");
    if (!run->finished) return fail(PMF_ESTATE, "run has not finished (call pmf_run_wait)");
    return PMF_OK;
}

extern "C" {

const char *pmf_last_error(void) { return g_err.c_str(); }
const char *pmf_version(void) { return "pmf-gb300 0.1 (sm_103a)"; }

pmf_status pmf_set_stream(void *stream)
{
    g_stream = reinterpret_cast<cudaStream_t>(stream);
    return PMF_OK;
}

pmf_status pmf_create_system(const pmf_system_desc *d, pmf_system **out)
{
    if (!d || !out) return fail(PMF_EINVAL, "pmf_create_system: null argument");
    *out = nullptr;
    auto sys = std::make_unique<pmf_system>();
    sys->model = d->model;
    sys->precision = d->precision;
    if (d->model == PMF_MODEL_1D_DOUBLEWELL) {
        if (!std::isfinite(d->dw_a) || !std::isfinite(d->x0)) return fail(PMF_EINVAL, "1D model: non-finite a or x0");
        sys->od.a = d->dw_a;
        sys->od.x0 = d->x0;
        if (pmf_status s = need_device()) return s;
        *out = sys.release();
        return PMF_OK;
    }
    if (d->model != PMF_MODEL_CHAIN) return fail(PMF_EINVAL, "unknown model");
    if (d->precision != PMF_FP32 && d->precision != PMF_FP64) return fail(PMF_EINVAL, "precision must be FP32 or FP64");
    if (d->n_chains < 1 || !d->n_beads) return fail(PMF_EINVAL, "chain model: n_chains >= 1 and n_beads[] required");
    if (!d->sigma || !d->epsilon || !d->charge || !d->mass || !d->dih_k || !d->dih_phase || !d->pos0)
        return fail(PMF_EINVAL, "chain model: a per-bead array is null");
    long long off = 0;
    std::vector<ChainHost> hosts;
    for (int c = 0; c < d->n_chains; ++c) {
        const int N = d->n_beads[c];
        if (N < 4 || N > 1024) return fail(PMF_EINVAL, "chain model: n_beads must be in [4, 1024]");
        ChainHost h;
        h.N = N;
        auto take = [&](const double *src, int per) { return std::vector<double>(src + off * per, src + (off + N) * per); };
        h.sigma = take(d->sigma, 1);
        h.epsilon = take(d->epsilon, 1);
        h.charge = take(d->charge, 1);
        h.mass = take(d->mass, 1);
        h.dih_k = take(d->dih_k, 3);
        h.dih_phase = take(d->dih_phase, 3);
        h.pos0 = take(d->pos0, 3);
        for (int b = 0; b < N; ++b) {
            if (!(h.mass[b] > 0) || !(h.epsilon[b] >= 0) || !std::isfinite(h.sigma[b]) || !std::isfinite(h.charge[b]))
                return fail(PMF_EINVAL, "chain model: invalid mass / epsilon / sigma / charge");
            for (int m = 0; m < 3; ++m) {
                if (!std::isfinite(h.pos0[3 * b + m])) return fail(PMF_EINVAL, "chain model: non-finite start state");
                const double ph = h.dih_phase[3 * b + m];
                if (b + 3 < N && h.dih_k[3 * b + m] != 0.0 && std::fabs(ph) > 1e-9 && std::fabs(std::fabs(ph) - M_PI) > 1e-9)
                    return fail(PMF_EINVAL, "chain model: dihedral phases must be 0 or pi");
            }
        }
        h.bond_k = d->bond_k;
        h.bond_r0 = d->bond_r0;
        h.angle_k = d->angle_k;
        h.angle_theta0 = d->angle_theta0;
        h.coulomb_k = d->coulomb_k;
        h.nonbonded = d->nonbonded;
        if (!std::isfinite(h.bond_k) || !std::isfinite(h.bond_r0) || !std::isfinite(h.angle_k) ||
            !std::isfinite(h.angle_theta0) || !std::isfinite(h.coulomb_k))
            return fail(PMF_EINVAL, "chain model: non-finite force-field constant");
        hosts.push_back(std::move(h));
        off += N;
    }
    if (pmf_status s = need_device()) return s;
    for (const ChainHost &h : hosts) {
        auto m = std::make_unique<ChainModel>();
        cudaError_t e = m->init(h, d->precision);
        if (e != cudaSuccess) return cuda_fail(e, "pmf_create_system");
        if (m->smem_bytes() > 227 * 1024 - 256) return fail(PMF_EINVAL, "chain too long for this precision (shared memory)");
        sys->chains.push_back(std::move(m));
    }
    *out = sys.release();
    return PMF_OK;
}

void pmf_destroy_system(pmf_system *sys) { delete sys; }

static pmf_status prepare_items(pmf_system *sys, const pmf_batch_item *items, int n_items, const pmf_run_params *p,
                                pmf_run **out, bool sequential = false)
{
    if (!sys || !items || !p || !out || n_items < 1) return fail(PMF_EINVAL, "pmf_run_prepare: null argument");
    *out = nullptr;
    long long total_w = 0;
    for (int it = 0; it < n_items; ++it) {
        const pmf_batch_item &I = items[it];
        if (!I.lambda || I.n_windows < 1) return fail(PMF_EINVAL, "each item needs lambda and n_windows >= 1");
        if (sys->model == PMF_MODEL_CHAIN && (I.chain < 0 || I.chain >= (int)sys->chains.size()))
            return fail(PMF_EINVAL, "chain index out of range");
        const double sgn = (I.n_windows > 1 && I.lambda[1] < I.lambda[0]) ? -1.0 : 1.0;
        for (int i = 0; i < I.n_windows; ++i) {
            if (!std::isfinite(I.lambda[i])) return fail(PMF_EINVAL, "lambda must be finite");
            if (i > 0 && !((I.lambda[i] - I.lambda[i - 1]) * sgn > 0))
                return fail(PMF_EINVAL, "lambda must be strictly monotone");
        }
        total_w += I.n_windows;
    }
    if (total_w > kMaxRunWindows) return fail(PMF_EINVAL, "a run holds at most 4096 windows");
    const int n_windows = (int)total_w;
    if (!(p->k > 0) || !(p->kT > 0) || !(p->dt > 0) || !(p->gamma >= 0) || !std::isfinite(p->k))
        return fail(PMF_EINVAL, "need k > 0, kT > 0, dt > 0, gamma >= 0");
    if (sys->model == PMF_MODEL_1D_DOUBLEWELL && !(p->gamma > 0)) return fail(PMF_EINVAL, "1D model needs gamma > 0");
    if (p->replicas < 1 || p->sample_stride < 1) return fail(PMF_EINVAL, "replicas >= 1 and sample_stride >= 1");
    if (p->replicas > 65535 || (long long)n_windows * p->replicas > (1LL << 31) - 1)
        return fail(PMF_EINVAL, "too many replicas (at most 65535 per window)");
    if (sequential && (n_items != 1 || p->n_steps_per_window))
        return fail(PMF_EINVAL, "the sequential protocol takes one path with one relaxation time for every window");
    auto run = std::make_unique<pmf_run>();
    run->sys = sys;
    run->sequential = sequential;
    run->chain = items[0].chain;
    run->n_windows = n_windows;
    run->replicas = p->replicas;
    run->stride = p->sample_stride;
    run->k = p->k;
    run->kT = p->kT;
    run->dt = p->dt;
    run->gamma = p->gamma;
    run->timeout_s = p->timeout_s;
    if (!(p->segment_wait_s >= 0) || !std::isfinite(p->segment_wait_s) || p->segment_wait_s > 1e6)
        return fail(PMF_EINVAL, "segment_wait_s must be in [0, 1e6]");
    run->segment_wait_s = p->segment_wait_s;
    run->seed = p->seed;
    run->uid_base = p->uid_base;
    size_t state_off = 0;
    int w0 = 0;
    for (int it = 0; it < n_items; ++it) {
        RunItem ri;
        ri.chain = sys->model == PMF_MODEL_CHAIN ? items[it].chain : 0;
        ri.w0 = w0;
        ri.nw = items[it].n_windows;
        ri.state_stride =
            sys->model == PMF_MODEL_CHAIN ? sys->chains[ri.chain]->state_bytes_per_replica() : 2 * sizeof(double);
        ri.state_off = state_off;
        state_off += ri.state_stride * (size_t)(sequential ? 1 : ri.nw) * p->replicas;
        run->items.push_back(ri);
        run->lambda.insert(run->lambda.end(), items[it].lambda, items[it].lambda + items[it].n_windows);
        w0 += ri.nw;
    }
    long long off = 0;
    for (int i = 0; i < n_windows; ++i) {
        const long long ns = p->n_steps_per_window ? p->n_steps_per_window[i] : p->n_steps;
        const long long ne = p->n_equil >= 0 ? p->n_equil : ns / 10;
        if (ns < 1 || ns >= (1LL << 32)) return fail(PMF_EINVAL, "n_steps must be in [1, 2^32)");
        if (ne < 0 || ne >= ns) return fail(PMF_EINVAL, "n_equil must be < n_steps");
        const long long T = (ns - ne) / p->sample_stride;
        if (T < 1) return fail(PMF_EINVAL, "each window needs at least one sample (n_steps - n_equil >= stride)");
        run->nsteps.push_back(ns);
        run->nequil.push_back(ne);
        run->tw.push_back(T);
        run->off.push_back(off);
        off += T * p->replicas;
        run->max_steps = std::max(run->max_steps, ns);
    }
    run->total = off;
    run->state_bytes = state_off;
    int max_nw = 0;
    for (const RunItem &ri : run->items) max_nw = std::max(max_nw, ri.nw);
    CK(upload(&run->d_lambda, run->lambda.data(), n_windows), "upload lambda");
    CK(upload(&run->d_nsteps, run->nsteps.data(), n_windows), "upload steps");
    CK(upload(&run->d_nequil, run->nequil.data(), n_windows), "upload equil");
    CK(upload(&run->d_off, run->off.data(), n_windows), "upload offsets");
    CK(upload(&run->d_tw, run->tw.data(), n_windows), "upload samples");
    CK(cudaMalloc(&run->d_x, sizeof(float) * run->total), "alloc samples");
    CK(cudaMalloc(&run->d_state, run->state_bytes), "alloc state");
    CK(cudaMalloc(&run->d_err, sizeof(int)), "alloc flag");
    CK(cudaMalloc(&run->d_scratch, reduce_scratch_bytes(max_nw, p->replicas)), "alloc scratch");
    CK(cudaMalloc(&run->d_res, sizeof(double) * kResFields * max_nw), "alloc results");
    CK(cudaEventCreateWithFlags(&run->done, cudaEventDisableTiming), "event");
    CK(cudaStreamCreateWithFlags(&run->cap, cudaStreamNonBlocking), "capture stream");
    if (sys->model == PMF_MODEL_1D_DOUBLEWELL) {
        // one noise block per item (a batch's items run concurrently)
        const long long sims = sequential ? p->replicas : (long long)n_windows * p->replicas;
        run->noise_steps = od1d_noise_steps((int)std::min<long long>(sims, 1 << 30));
        CK(cudaMalloc(&run->d_noise, sizeof(double) * (size_t)run->noise_steps * sims), "alloc noise");
    }
    if (sys->model == PMF_MODEL_CHAIN) {
        CK(cudaHostAlloc(&run->h_abort, sizeof(int), cudaHostAllocMapped), "alloc stop flag");
        *(volatile int *)run->h_abort = 0;
        CK(cudaHostGetDevicePointer(&run->d_abort, run->h_abort, 0), "map stop flag");
    }
    if (n_items == 1 && sys->model == PMF_MODEL_CHAIN) {
        CK(cudaMalloc(&run->d_queue, sizeof(unsigned long long)), "alloc queue");
        CK(cudaMalloc(&run->d_done, sizeof(int) * (size_t)n_windows * p->replicas), "alloc segment counters");
    }
    if (n_items > 1 && sys->model == PMF_MODEL_CHAIN && !sequential) {
        bool packable = true;
        for (const RunItem &ri : run->items)
            packable = packable && sys->chains[ri.chain]->precision() != PMF_FP64 &&
                       pack_team_choice(*sys->chains[ri.chain], 0) > 0;
        run->batch_mode = packable ? 1 : 0;
    }
    const int n_branch = std::min(n_items, kMaxBranches);
    if (n_branch > 1) {
        run->fork_ev.assign(1 + n_branch, nullptr);
        run->branch.assign(n_branch, nullptr);
        for (auto &e : run->fork_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "fork event");
        for (auto &b : run->branch) CK(cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking), "branch stream");
    }
    *out = run.release();
    return PMF_OK;
}

pmf_status pmf_run_prepare(pmf_system *sys, const double *lambda, int n_windows, const pmf_run_params *p,
                           pmf_run **out)
{
    if (!p) return fail(PMF_EINVAL, "pmf_run_prepare: null params");
    if (n_windows < 1 || n_windows > 1024) return fail(PMF_EINVAL, "n_windows must be in [1, 1024]");
    pmf_batch_item it{p->chain, n_windows, lambda};
    return prepare_items(sys, &it, 1, p, out);
}

pmf_status pmf_run_batch_prepare(pmf_system *sys, const pmf_batch_item *items, int n_items, const pmf_run_params *p,
                                 pmf_run **out)
{
    return prepare_items(sys, items, n_items, p, out);
}

pmf_status pmf_run_prepare_sequential(pmf_system *sys, const double *lambda, int n_windows, const pmf_run_params *p,
                                      pmf_run **out)
{
    if (!p) return fail(PMF_EINVAL, "pmf_run_prepare_sequential: null params");
    if (n_windows < 1 || n_windows > 1024) return fail(PMF_EINVAL, "n_windows must be in [1, 1024]");
    if ((long long)n_windows * p->n_steps >= (1LL << 32))
        return fail(PMF_EINVAL, "the sequential run's total step count must be below 2^32");
    pmf_batch_item it{p->chain, n_windows, lambda};
    return prepare_items(sys, &it, 1, p, out, true);
}

// Modelled cost of one replica of an item: pair interactions x steps.
static double item_cost(const pmf_run *run, const RunItem &ri)
{
    const double N = run->sys->model == PMF_MODEL_CHAIN ? run->sys->chains[ri.chain]->n_beads() : 1.0;
    long long steps = 0;
    for (int w = ri.w0; w < ri.w0 + ri.nw; ++w) steps = std::max(steps, run->nsteps[w]);
    return (N * N * 0.5 + 40.0 * N) * (double)steps;
}

// Enqueue every launch of one item on stream st: one launch per 1e5-step
// chunk (chain model) over the item's nw x replicas CTAs; state carries over
// between chunks in device memory.
// The launch fields of one item of the run (one-CTA-per-replica form).
static RunLaunch item_launch(const pmf_run *run, const RunItem &ri)
{
    RunLaunch L;
    L.state = static_cast<char *>(run->d_state) + ri.state_off;
    L.xout = run->d_x;
    L.lambda = run->d_lambda + ri.w0;
    L.nsteps_w = run->d_nsteps + ri.w0;
    L.nequil_w = run->d_nequil + ri.w0;
    L.off_w = run->d_off + ri.w0;
    L.tw = run->d_tw + ri.w0;
    L.err = run->d_err;
    L.start = run->d_start;
    L.queue = run->d_queue;  // set for single-item chain runs only
    L.done = run->d_done;
    L.queue_start = run->queue_start;
    L.wait_ns = (unsigned long long)(run->segment_wait_s * 1e9);
    L.abort = run->d_abort;
    L.wout = run->d_w;       // set for pulled runs only
    L.smd_vdt = run->smd_vdt;
    // 1D runs: this item's block of the noise buffer
    L.noise = run->d_noise ? run->d_noise + (size_t)run->noise_steps * ri.w0 * run->replicas : nullptr;
    L.noise_steps = run->noise_steps;
    L.replicas = run->replicas;
    L.stride = run->stride;
    L.uid_base = run->uid_base + (uint32_t)(ri.w0 * run->replicas);
    L.seed = run->seed;
    L.k = run->k;
    L.kT = run->kT;
    L.dt = run->dt;
    L.gamma = run->gamma;
    L.n_blocks = ri.nw * run->replicas;
    return L;
}

// Enqueue every launch of one item on stream st: one launch per 1e5-step
// chunk (chain model) over the item's nw x replicas CTAs; state carries over
// between chunks in device memory.
static cudaError_t enqueue_item(pmf_run *run, const RunItem &ri, cudaStream_t st)
{
    RunLaunch L = item_launch(run, ri);
    if (run->sequential) {
        // one launch: each replica visits every window, nsteps[0] steps each
        L.sequential = true;
        L.window_steps = run->nsteps[0];
        L.uid_base = run->uid_base;
        L.n_blocks = run->replicas;
        L.step_begin = 0;
        L.step_end = run->nsteps[0] * ri.nw;
        return run->sys->model == PMF_MODEL_CHAIN ? run->sys->chains[ri.chain]->launch(L, st)
                                                  : od1d_launch(run->sys->od, L, run->replicas, st);
    }
    const int n_rep = ri.nw * run->replicas;
    L.n_blocks = n_rep;
    long long max_steps = 0;
    for (int w = ri.w0; w < ri.w0 + ri.nw; ++w) max_steps = std::max(max_steps, run->nsteps[w]);
    if (run->probe_steps > 0) max_steps = std::min(max_steps, run->probe_steps);
    const long long chunk = run->sys->model == PMF_MODEL_CHAIN ? 100000 : (1LL << 40);
    for (long long s0 = 0; s0 < max_steps; s0 += chunk) {
        L.step_begin = s0;
        L.step_end = std::min(max_steps, s0 + chunk);
        cudaError_t e = run->sys->model == PMF_MODEL_CHAIN ? run->sys->chains[ri.chain]->launch(L, st)
                                                          : od1d_launch(run->sys->od, L, n_rep, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The packed launch plan of a batched FP32 chain run (team sizes from the
// run's shift), built on first use.
static cudaError_t ensure_pack(pmf_run *run)
{
    if (run->pack) return cudaSuccess;
    std::vector<PackItemSpec> specs;
    std::vector<int> teams;
    int seg = 1000;
    for (const RunItem &ri : run->items) {
        ChainModel *m = run->sys->chains[ri.chain].get();
        const int G = pack_team_choice(*m, run->pack_shift);
        if (G < 0) return cudaErrorInvalidValue;
        specs.push_back(PackItemSpec{m, item_launch(run, ri)});
        teams.push_back(G);
        seg = m->seg_steps();
    }
    return pack_plan_create(specs, teams, seg, &run->pack);
}

// Enqueue the run's whole launch sequence on stream st (the capture stream).
// A packed batch is one persistent launch per chunk.  Otherwise a batch
// forks into independent branches, one chain of launches per item,
// so that the items' kernels run concurrently and the block scheduler fills
// the SMs; items are issued costliest first (longest CTAs start first) and
// dealt to branches by least accumulated cost.
static cudaError_t enqueue_run(pmf_run *run, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(run->d_err, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (run->batch_mode == 1) {
        // one packed persistent launch per 1e5-step chunk for the whole batch
        if ((e = ensure_pack(run)) != cudaSuccess) return e;
        long long max_steps = run->max_steps;
        if (run->probe_steps > 0) max_steps = std::min(max_steps, run->probe_steps);
        for (long long s0 = 0; s0 < max_steps; s0 += 100000)
            if ((e = pack_plan_launch(run->pack, s0, std::min(max_steps, s0 + 100000), st)) != cudaSuccess) return e;
        return cudaSuccess;
    }
    if (run->branch.empty()) {
        for (const RunItem &ri : run->items)
            if ((e = enqueue_item(run, ri, st)) != cudaSuccess) return e;
        return cudaSuccess;
    }
    const int nb = (int)run->branch.size();
    if ((e = cudaEventRecord(run->fork_ev[0], st)) != cudaSuccess) return e;
    for (int b = 0; b < nb; ++b)
        if ((e = cudaStreamWaitEvent(run->branch[b], run->fork_ev[0], 0)) != cudaSuccess) return e;
    std::vector<int> order(run->items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::vector<double> cost(order.size());
    for (size_t i = 0; i < order.size(); ++i) cost[i] = item_cost(run, run->items[i]);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> load(nb, 0.0);
    for (int i : order) {
        const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[b] += cost[i] * run->items[i].nw;
        if ((e = enqueue_item(run, run->items[i], run->branch[b])) != cudaSuccess) return e;
    }
    for (int b = 0; b < nb; ++b) {
        if ((e = cudaEventRecord(run->fork_ev[1 + b], run->branch[b])) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(st, run->fork_ev[1 + b], 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

pmf_status pmf_run_launch(pmf_run *run)
{
    if (!run) return fail(PMF_EINVAL, "pmf_run_launch: null run");
    if (run->d_start && run->items.size() > 1) return fail(PMF_EINVAL, "seeded starts need a single-item run");
    // the whole launch sequence is captured once into a CUDA graph and
    // replayed; it is re-captured when a chain's work schedule was rebuilt
    // (pmf_chain_set_warps / pmf_chain_autotune) since the capture
    std::vector<unsigned> gen;
    for (const RunItem &ri : run->items)
        gen.push_back(run->sys->model == PMF_MODEL_CHAIN ? run->sys->chains[ri.chain]->generation() : 0u);
    if (!run->graph || gen != run->graph_gen) {
        if (run->graph) {
            cudaGraphExecDestroy(run->graph);
            run->graph = nullptr;
        }
        if (run->pack && gen != run->graph_gen) {  // a schedule was rebuilt: so is the plan
            pack_plan_destroy(run->pack);
            run->pack = nullptr;
        }
        CK(cudaStreamBeginCapture(run->cap, cudaStreamCaptureModeRelaxed), "begin capture");
        cudaError_t e = enqueue_run(run, run->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(run->cap, &g);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(e, "capture run");
        }
        if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
        e = cudaGraphInstantiate(&run->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "instantiate graph");
        run->graph_gen = gen;
    }
    if (run->h_abort) *(volatile int *)run->h_abort = 0;
    CK(cudaGraphLaunch(run->graph, g_stream), "graph launch");
    CK(cudaEventRecord(run->done, g_stream), "record");
    run->launched = true;
    run->finished = false;
    run->reduced = false;
    return PMF_OK;
}

pmf_status pmf_run_wait(pmf_run *run)
{
    if (!run || !run->launched) return fail(PMF_ESTATE, "pmf_run_wait: run not launched");
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t q = cudaEventQuery(run->done);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return cuda_fail(q, "run");
        if (run->timeout_s > 0) {
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (el > run->timeout_s) {
                // ask the persistent chain launches to stop at their next
                // work item, then wait for the kernels in flight to drain so
                // that no kernel of this run still uses its buffers
                if (run->h_abort) *(volatile int *)run->h_abort = 1;
                cudaError_t e = cudaEventSynchronize(run->done);
                if (e != cudaSuccess) return cuda_fail(e, "run (stopping after timeout_s)");
                run->finished = false;
                return fail(PMF_ETIMEOUT, "run exceeded timeout_s and was stopped (its samples are incomplete)");
            }
        }
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    int err = 0;
    CK(cudaMemcpy(&err, run->d_err, sizeof(int), cudaMemcpyDeviceToHost), "read flag");
    run->finished = true;
    if (err & kErrTimeout) {
        run->finished = false;
        return fail(PMF_ETIMEOUT, "a persistent segment waited longer than segment_wait_s for the replica's "
                                  "previous segment (the run stopped; its samples are incomplete)");
    }
    if (err & kErrNonFinite) return fail(PMF_ENUMERIC, "a trajectory became non-finite");
    if (err) return fail(PMF_ECUDA, "device error flag " + std::to_string(err));
    return PMF_OK;
}

pmf_status pmf_run_prepare_smd(pmf_system *sys, double lambda1, double velocity, const pmf_run_params *p,
                               pmf_run **out)
{
    if (!p || !out) return fail(PMF_EINVAL, "pmf_run_prepare_smd: null argument");
    if (!std::isfinite(lambda1) || !std::isfinite(velocity)) return fail(PMF_EINVAL, "lambda1 and velocity must be finite");
    if (p->n_steps_per_window) return fail(PMF_EINVAL, "pmf_run_prepare_smd: one pull, no per-window steps");
    if (pmf_status st = pmf_run_prepare(sys, &lambda1, 1, p, out)) return st;
    pmf_run *run = *out;
    run->smd_vdt = velocity * p->dt;
    cudaError_t e = cudaMalloc(&run->d_w, sizeof(double) * (size_t)run->total);
    if (e != cudaSuccess) {
        pmf_destroy_run(run);
        *out = nullptr;
        return cuda_fail(e, "alloc work records");
    }
    return PMF_OK;
}

pmf_status pmf_smd_work(const pmf_run *run, double *out, size_t capacity, size_t *n_written)
{
    if (pmf_status s = need_finished(run)) return s;
    if (!run->d_w) return fail(PMF_EINVAL, "pmf_smd_work: not a pulled run");
    if (n_written) *n_written = (size_t)run->total;
    if (!out || capacity < (size_t)run->total) return fail(PMF_EINVAL, "pmf_smd_work: capacity too small");
    CK(cudaMemcpyAsync(out, run->d_w, sizeof(double) * run->total, cudaMemcpyDeviceToHost, g_stream), "copy");
    CK(cudaStreamSynchronize(g_stream), "sync");
    return PMF_OK;
}

pmf_status pmf_smd_free_energy(const pmf_run *run, double *lambda, double *dF_JE, double *dF_cumulant,
                               double *W_mean, double *W_var, double *mean_x, int capacity)
{
    if (pmf_status s = need_finished(run)) return s;
    if (!run->d_w) return fail(PMF_EINVAL, "pmf_smd_free_energy: not a pulled run");
    const long long T = run->tw[0];
    if (capacity < T) return fail(PMF_EINVAL, "pmf_smd_free_energy: capacity smaller than the records");
    double *d_out = nullptr;
    CK(cudaMalloc(&d_out, sizeof(double) * 5 * (size_t)T), "alloc");
    cudaError_t e = smd_stats_launch(run->d_w, run->d_x, run->replicas, T, run->kT, d_out, g_stream);
    std::vector<double> h(5 * (size_t)T);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), d_out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, g_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
    cudaFree(d_out);
    if (e != cudaSuccess) return cuda_fail(e, "pmf_smd_free_energy");
    double *dst[5] = {dF_JE, dF_cumulant, W_mean, W_var, mean_x};
    for (int q = 0; q < 5; ++q)
        if (dst[q]) std::memcpy(dst[q], h.data() + (size_t)q * T, sizeof(double) * T);
    if (lambda)
        for (long long j = 0; j < T; ++j)
            lambda[j] = run->lambda[0] + run->smd_vdt * (double)((j + 1) * run->stride);
    return PMF_OK;
}

pmf_status pmf_run_prepare_seeded(pmf_system *sys, const double *lambda, int n_windows, const pmf_run_params *p,
                                  const double *start, pmf_run **out)
{
    if (!start) return fail(PMF_EINVAL, "pmf_run_prepare_seeded: null start");
    pmf_status s = pmf_run_prepare(sys, lambda, n_windows, p, out);
    if (s != PMF_OK) return s;
    pmf_run *run = *out;
    const size_t n_rep = (size_t)n_windows * p->replicas;
    const size_t per = sys->model == PMF_MODEL_CHAIN ? (size_t)sys->chains[p->chain]->n_beads() * 3 : 1;
    for (size_t i = 0; i < n_rep * per; ++i)
        if (!std::isfinite(start[i])) {
            pmf_destroy_run(run);
            *out = nullptr;
            return fail(PMF_EINVAL, "pmf_run_prepare_seeded: non-finite start state");
        }
    cudaError_t e = upload(&run->d_start, start, n_rep * per);
    if (e != cudaSuccess) {
        pmf_destroy_run(run);
        *out = nullptr;
        return cuda_fail(e, "upload start states");
    }
    return PMF_OK;
}

pmf_status pmf_run_windows(pmf_system *sys, const double *lambda, int n_windows, const pmf_run_params *p,
                           pmf_run **out)
{
    pmf_status s = pmf_run_prepare(sys, lambda, n_windows, p, out);
    if (s != PMF_OK) return s;
    if ((s = pmf_run_launch(*out)) != PMF_OK) return s;
    return pmf_run_wait(*out);
}

void pmf_destroy_run(pmf_run *run) { delete run; }

pmf_status pmf_get_run_info(const pmf_run *run, pmf_run_info *info)
{
    if (!run || !info) return fail(PMF_EINVAL, "pmf_get_run_info: null argument");
    std::memset(info, 0, sizeof(*info));
    info->n_windows = run->n_windows;
    info->replicas = run->replicas;
    info->total_samples = run->total;
    for (int i = 0; i < run->n_windows; ++i) {
        info->samples_per_window[i] = run->tw[i];
        info->sample_offset[i] = run->off[i];
    }
    return PMF_OK;
}


pmf_status pmf_x_samples(const pmf_run *run, float *out, size_t capacity, size_t *n_written)
{
    if (pmf_status s = need_finished(run)) return s;
    if (n_written) *n_written = (size_t)run->total;
    if (!out || capacity < (size_t)run->total) return fail(PMF_EINVAL, "pmf_x_samples: capacity too small");
    CK(cudaMemcpyAsync(out, run->d_x, sizeof(float) * run->total, cudaMemcpyDeviceToHost, g_stream), "copy samples");
    CK(cudaStreamSynchronize(g_stream), "sync");
    return PMF_OK;
}

static ReduceLayout layout_of(const pmf_run *run)
{
    ReduceLayout L;
    L.x = run->d_x;
    L.lambda = run->d_lambda;
    L.off_w = run->d_off;
    L.tw = run->d_tw;
    L.n_windows = run->n_windows;
    L.replicas = run->replicas;
    L.k = run->k;
    L.kT = run->kT;
    return L;
}

pmf_status pmf_work_samples(const pmf_run *run, int mode, double *out, size_t capacity, size_t *n_written)
{
    if (pmf_status s = need_finished(run)) return s;
    if (run->items.size() != 1) return fail(PMF_EINVAL, "pmf_work_samples: single-item runs only");
    long long need = 0;
    if (mode == PMF_WORK_PER_WINDOW_INCREMENT) {
        need = run->off[run->n_windows - 1];
    } else if (mode == PMF_WORK_PAIRED_CUMULATIVE) {
        for (int i = 1; i < run->n_windows; ++i)
            if (run->tw[i] != run->tw[0]) return fail(PMF_EINVAL, "paired work needs equal samples per window");
        need = (long long)(run->n_windows - 1) * run->replicas * run->tw[0];
    } else {
        return fail(PMF_EINVAL, "unknown work mode");
    }
    if (n_written) *n_written = (size_t)need;
    if (!out || capacity < (size_t)need) return fail(PMF_EINVAL, "pmf_work_samples: capacity too small");
    double *d = nullptr;
    CK(cudaMalloc(&d, sizeof(double) * (need ? need : 1)), "alloc work");
    cudaError_t e = work_samples_launch(layout_of(run), mode, run->tw[0], d, g_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, sizeof(double) * need, cudaMemcpyDeviceToHost, g_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "work samples");
    return PMF_OK;
}

static pmf_status copy_result(const double *host, int s, pmf_free_energy_result *res)
{
    if (res->capacity < s) return fail(PMF_EINVAL, "result capacity smaller than n_windows");
    double *dst[kResFields] = {res->lambda, res->dF_JE, res->dF_fluct, res->dF_G, res->dF_com, res->uncertainty,
                               res->se_JE, res->se_fluct, res->var_ZW, res->W_mean, res->acc_force, res->mean_x,
                               res->var_x, res->gamma2};
    for (int q = 0; q < kResFields; ++q)
        if (dst[q]) std::memcpy(dst[q], host + (size_t)q * s, sizeof(double) * s);
    return PMF_OK;
}

static ReduceLayout item_layout(const pmf_run *run, int item)
{
    ReduceLayout L = layout_of(run);
    const RunItem &ri = run->items[item];
    L.lambda = run->d_lambda + ri.w0;
    L.off_w = run->d_off + ri.w0;
    L.tw = run->d_tw + ri.w0;
    L.n_windows = ri.nw;
    return L;
}

pmf_status pmf_free_energy_item(const pmf_run *run, int item, pmf_free_energy_result *res)
{
    if (pmf_status s = need_finished(run)) return s;
    if (!res || item < 0 || item >= (int)run->items.size()) return fail(PMF_EINVAL, "pmf_free_energy_item: bad item");
    const int nw = run->items[item].nw;
    if (nw < 2) return fail(PMF_EINVAL, "pmf_free_energy_item: the item needs two windows");
    if (res->capacity < nw) return fail(PMF_EINVAL, "result capacity smaller than the item's windows");
    cudaError_t e = reduce_launch(item_layout(run, item), run->d_scratch, run->d_res, g_stream);
    if (e != cudaSuccess) return cuda_fail(e, "reduce");
    const_cast<pmf_run *>(run)->reduced = false;  // d_res now holds this item
    std::vector<double> h((size_t)kResFields * nw);
    CK(cudaMemcpyAsync(h.data(), run->d_res, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, g_stream), "copy");
    CK(cudaStreamSynchronize(g_stream), "sync");
    return copy_result(h.data(), nw, res);
}

pmf_status pmf_run_set_batch_launch(pmf_run *run, int mode, int shift)
{
    if (!run) return fail(PMF_EINVAL, "null run");
    if (mode != PMF_BATCH_GRAPH && mode != PMF_BATCH_PACKED) return fail(PMF_EINVAL, "unknown batch mode");
    if (shift < 0 || shift > 2) return fail(PMF_EINVAL, "packing policy must be 0, 1 or 2");
    if (run->launched && !run->finished && cudaEventQuery(run->done) == cudaErrorNotReady)
        return fail(PMF_ESTATE, "pmf_run_set_batch_launch: the run is still in flight");
    if (mode == PMF_BATCH_PACKED) {
        if (run->sys->model != PMF_MODEL_CHAIN || run->sequential || run->d_w || run->d_start)
            return fail(PMF_EINVAL, "packed launches: chain window runs only");
        for (const RunItem &ri : run->items) {
            const ChainModel &m = *run->sys->chains[ri.chain];
            if (m.precision() == PMF_FP64 || pack_team_choice(m, shift) < 0)
                return fail(PMF_EINVAL, "packed launches: FP32 chains that fit a packed CTA only");
        }
    }
    if (mode != run->batch_mode || shift != run->pack_shift) {
        run->batch_mode = mode;
        run->pack_shift = shift;
        pack_plan_destroy(run->pack);
        run->pack = nullptr;
        if (run->graph) {
            cudaGraphExecDestroy(run->graph);
            run->graph = nullptr;
        }
    }
    return PMF_OK;
}

pmf_status pmf_run_get_batch_launch(pmf_run *run, int *mode, int *shift, int *packs, int *ctas, int *teams,
                                    int capacity)
{
    if (!run) return fail(PMF_EINVAL, "null run");
    if (mode) *mode = run->batch_mode;
    if (shift) *shift = run->pack_shift;
    if (run->batch_mode == PMF_BATCH_PACKED) {
        cudaError_t e = ensure_pack(run);
        if (e != cudaSuccess) return cuda_fail(e, "pmf_run_get_batch_launch");
    }
    if (packs) *packs = pack_plan_packs(run->pack);
    if (ctas) *ctas = pack_plan_grid(run->pack);
    if (teams) {
        if (capacity < (int)run->items.size()) return fail(PMF_EINVAL, "teams capacity smaller than the items");
        for (size_t m = 0; m < run->items.size(); ++m)
            teams[m] = run->batch_mode == PMF_BATCH_PACKED
                           ? pack_team_choice(*run->sys->chains[run->items[m].chain], run->pack_shift)
                           : 0;
    }
    return PMF_OK;
}

pmf_status pmf_run_batch_autotune(pmf_run *run, int64_t probe_steps, double *best_ms)
{
    if (!run || probe_steps < 1) return fail(PMF_EINVAL, "pmf_run_batch_autotune: bad argument");
    if (run->items.size() < 2 || run->sys->model != PMF_MODEL_CHAIN)
        return fail(PMF_EINVAL, "pmf_run_batch_autotune: batched chain runs only");
    struct Cand {
        int mode, shift;
    };
    std::vector<Cand> cands = {{PMF_BATCH_GRAPH, 0}};
    for (int sh = 0; sh <= 2; ++sh) {
        bool ok = true;
        for (const RunItem &ri : run->items) {
            const ChainModel &m = *run->sys->chains[ri.chain];
            ok = ok && m.precision() != PMF_FP64 && pack_team_choice(m, sh) > 0;
        }
        if (!ok) continue;
        bool dup = false;
        for (const Cand &c : cands) {
            if (c.mode != PMF_BATCH_PACKED) continue;
            bool same = true;
            for (const RunItem &ri : run->items) {
                const ChainModel &m = *run->sys->chains[ri.chain];
                same = same && pack_team_choice(m, sh) == pack_team_choice(m, c.shift);
            }
            dup = dup || same;
        }
        if (!dup) cands.push_back(Cand{PMF_BATCH_PACKED, sh});
    }
    const int mode0 = run->batch_mode, shift0 = run->pack_shift;
    Cand best{mode0, shift0};
    double best_t = 1e300;
    GpuTimer timer;
    run->probe_steps = probe_steps;
    pmf_status st = PMF_OK;
    for (const Cand &c : cands) {
        if ((st = pmf_run_set_batch_launch(run, c.mode, c.shift)) != PMF_OK) break;
        if ((st = pmf_run_launch(run)) != PMF_OK || (st = pmf_run_wait(run)) != PMF_OK) break;  // warm-up, capture
        double t = 1e300;
        for (int rep = 0; rep < 2 && st == PMF_OK; ++rep) {
            const double before = timer.ms;
            timer.start();
            if ((st = pmf_run_launch(run)) != PMF_OK) break;
            cudaError_t e = timer.stop();
            if (e != cudaSuccess) { st = cuda_fail(e, "autotune timer"); break; }
            if ((st = pmf_run_wait(run)) != PMF_OK) break;
            t = std::min(t, timer.ms - before);
        }
        if (st != PMF_OK) break;
        if (t < best_t) {
            best_t = t;
            best = c;
        }
    }
    run->probe_steps = 0;
    // the probes overwrote the run's samples and states: the next launch
    // starts from x_o again; the captured probe launches are dropped
    if (run->graph) {
        cudaGraphExecDestroy(run->graph);
        run->graph = nullptr;
    }
    run->finished = false;
    if (st != PMF_OK) return st;
    if (pmf_status s2 = pmf_run_set_batch_launch(run, best.mode, best.shift)) return s2;
    if (best_ms) *best_ms = best_t;
    return PMF_OK;
}

pmf_status pmf_run_set_queue_start(pmf_run *run, int64_t first_item)
{
    if (!run) return fail(PMF_EINVAL, "null run");
    if (!run->d_queue || run->sequential || run->items.size() != 1)
        return fail(PMF_EINVAL, "pmf_run_set_queue_start: single-item chain runs with the persistent launch only");
    if (first_item < 0) return fail(PMF_EINVAL, "pmf_run_set_queue_start: first_item must be >= 0");
    if (run->launched && !run->finished && cudaEventQuery(run->done) == cudaErrorNotReady)
        return fail(PMF_ESTATE, "pmf_run_set_queue_start: the run is still in flight");
    run->queue_start = first_item;
    if (run->graph) {  // the offset is a kernel argument: capture the launches again
        cudaGraphExecDestroy(run->graph);
        run->graph = nullptr;
    }
    return PMF_OK;
}

pmf_status pmf_run_reduce(pmf_run *run)
{
    if (!run) return fail(PMF_EINVAL, "null run");
    if (!run->launched) return fail(PMF_ESTATE, "pmf_run_reduce: run not launched");
    if (run->items.size() != 1) return fail(PMF_EINVAL, "pmf_run_reduce: use pmf_free_energy_item on batch runs");
    cudaError_t e = reduce_launch(layout_of(run), run->d_scratch, run->d_res, g_stream);
    if (e != cudaSuccess) return cuda_fail(e, "reduce");
    run->reduced = true;
    return PMF_OK;
}

pmf_status pmf_free_energy(const pmf_run *run, pmf_free_energy_result *res)
{
    if (pmf_status s = need_finished(run)) return s;
    if (!res) return fail(PMF_EINVAL, "null result");
    if (run->items.size() != 1) return fail(PMF_EINVAL, "pmf_free_energy: use pmf_free_energy_item on batch runs");
    if (res->capacity < run->n_windows) return fail(PMF_EINVAL, "result capacity smaller than n_windows");
    if (!run->reduced) {
        cudaError_t e = reduce_launch(layout_of(run), run->d_scratch, run->d_res, g_stream);
        if (e != cudaSuccess) return cuda_fail(e, "reduce");
        const_cast<pmf_run *>(run)->reduced = true;
    }
    std::vector<double> h((size_t)kResFields * run->n_windows);
    CK(cudaMemcpyAsync(h.data(), run->d_res, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, g_stream), "copy");
    CK(cudaStreamSynchronize(g_stream), "sync");
    return copy_result(h.data(), run->n_windows, res);
}

pmf_status pmf_work_distributions(const pmf_run *run, const pmf_hist_params *hp, double *omega,
                                  size_t omega_capacity, double *dF_JE, double *var_ZW, double *lost)
{
    if (pmf_status s = need_finished(run)) return s;
    if (!hp) return fail(PMF_EINVAL, "pmf_work_distributions: null parameters");
    if (run->items.size() != 1) return fail(PMF_EINVAL, "pmf_work_distributions: single-item runs only");
    if (!(hp->dx > 0) || !(hp->dw > 0) || !std::isfinite(hp->x_lo) || hp->n_x < 1 || hp->n_x > (1 << 26) ||
        hp->M < 1 || hp->M > (1 << 24))
        return fail(PMF_EINVAL, "pmf_work_distributions: bad bins");
    const int s = run->n_windows;
    const long long M = hp->M, nb = 2 * M + 1;
    if (omega && omega_capacity < (size_t)s * nb) return fail(PMF_EINVAL, "pmf_work_distributions: omega too small");
    struct Tmp {
        unsigned long long *cnt = nullptr, *outside = nullptr;
        int *jmin = nullptr, *jmax = nullptr;
        double *om = nullptr, *g = nullptr, *stats = nullptr;
        long long *sup = nullptr;
        ~Tmp() { cudaFree(cnt); cudaFree(outside); cudaFree(jmin); cudaFree(jmax); cudaFree(om); cudaFree(g);
                 cudaFree(stats); cudaFree(sup); }
    } t;
    CK(cudaMalloc(&t.cnt, sizeof(unsigned long long) * (size_t)s * hp->n_x), "alloc counts");
    CK(cudaMalloc(&t.outside, sizeof(unsigned long long) * s), "alloc");
    CK(cudaMalloc(&t.jmin, sizeof(int) * s), "alloc");
    CK(cudaMalloc(&t.jmax, sizeof(int) * s), "alloc");
    CK(cudaMalloc(&t.om, sizeof(double) * (size_t)s * nb), "alloc omega");
    CK(cudaMalloc(&t.stats, sizeof(double) * 4 * s), "alloc");
    CK(cudaMalloc(&t.sup, sizeof(long long) * 2 * s), "alloc");
    CK(cudaMemsetAsync(t.cnt, 0, sizeof(unsigned long long) * (size_t)s * hp->n_x, g_stream), "clear");
    CK(cudaMemsetAsync(t.outside, 0, sizeof(unsigned long long) * s, g_stream), "clear");
    CK(cudaMemsetAsync(t.jmin, 0x7f, sizeof(int) * s, g_stream), "clear");
    CK(cudaMemsetAsync(t.jmax, 0xff, sizeof(int) * s, g_stream), "clear");
    CK(cudaMemsetAsync(t.om, 0, sizeof(double) * (size_t)s * nb, g_stream), "clear");
    CK(hist_count_launch(run->d_x, run->d_off, run->d_tw, s, run->replicas, hp->x_lo, hp->dx, hp->n_x, t.cnt, t.outside,
                         t.jmin, t.jmax, g_stream), "count");
    std::vector<int> jmin(s), jmax(s);
    CK(cudaMemcpyAsync(jmin.data(), t.jmin, sizeof(int) * s, cudaMemcpyDeviceToHost, g_stream), "copy");
    CK(cudaMemcpyAsync(jmax.data(), t.jmax, sizeof(int) * s, cudaMemcpyDeviceToHost, g_stream), "copy");
    CK(cudaStreamSynchronize(g_stream), "sync");
    for (int i = 0; i + 1 < s; ++i)
        if (jmax[i] < jmin[i]) return fail(PMF_EINVAL, "pmf_work_distributions: a window has no sample in the x range");
    // supports: Omega_1 at b = 0, then Omega_{i+1} = Omega_i * g_i
    std::vector<long long> sup(2 * (size_t)s);
    std::vector<HistStep> steps(s > 1 ? s - 1 : 0);
    sup[0] = sup[1] = 0;
    long long max_ng = 1;
    for (int i = 0; i + 1 < s; ++i) {
        HistStep &h = steps[i];
        h.x_lo = hp->x_lo;
        h.dx = hp->dx;
        h.dw = hp->dw;
        h.hk = 0.5 * run->k;
        h.d = run->lambda[i + 1] - run->lambda[i];
        h.lsum = run->lambda[i + 1] + run->lambda[i];
        h.left_edge = hp->left_edge ? 1 : 0;
        h.jmin = jmin[i];
        h.jmax = jmax[i];
        const long long a = hist_shift_host(h, h.jmin), b = hist_shift_host(h, h.jmax);
        h.gmin = std::min(a, b) - 1;
        h.gmax = std::max(a, b) + 1;
        max_ng = std::max(max_ng, h.gmax - h.gmin + 1);
        long long lo = sup[2 * i] + h.gmin, hi = sup[2 * i + 1] + h.gmax;
        if (h.left_edge) {
            lo = std::min(lo, -1LL);
            hi = std::max(hi, 1LL);
        }
        sup[2 * (i + 1)] = std::max(lo, -M);
        sup[2 * (i + 1) + 1] = std::min(hi, M);
    }
    CK(cudaMalloc(&t.g, sizeof(double) * (size_t)max_ng), "alloc shifts");
    const double one = 1.0;
    CK(cudaMemcpyAsync(t.om + M, &one, sizeof(double), cudaMemcpyHostToDevice, g_stream), "init");
    for (int i = 0; i + 1 < s; ++i) {
        const double inv_n = 1.0 / (double)(run->tw[i] * run->replicas);
        CK(hist_step_launch(steps[i], t.cnt + (size_t)i * hp->n_x, inv_n, t.g, t.om + (size_t)i * nb, sup[2 * i],
                            sup[2 * i + 1], t.om + (size_t)(i + 1) * nb, sup[2 * (i + 1)], sup[2 * (i + 1) + 1], M,
                            g_stream),
           "convolution");
    }
    CK(cudaMemcpyAsync(t.sup, sup.data(), sizeof(long long) * 2 * s, cudaMemcpyHostToDevice, g_stream), "upload");
    CK(hist_stats_launch(t.om, s, M, hp->dw, run->kT, t.sup, t.stats, g_stream), "stats");
    std::vector<double> st(4 * (size_t)s);
    CK(cudaMemcpyAsync(st.data(), t.stats, sizeof(double) * st.size(), cudaMemcpyDeviceToHost, g_stream), "copy");
    if (omega) CK(cudaMemcpyAsync(omega, t.om, sizeof(double) * (size_t)s * nb, cudaMemcpyDeviceToHost, g_stream), "copy");
    CK(cudaStreamSynchronize(g_stream), "sync");
    for (int i = 0; i < s; ++i) {
        if (dF_JE) dF_JE[i] = st[4 * i];
        if (var_ZW) var_ZW[i] = st[4 * i + 1];
        if (lost) lost[i] = i == 0 ? 0.0 : std::max(0.0, 1.0 - st[4 * i + 2]);
    }
    return PMF_OK;
}

pmf_status pmf_run_partials(const pmf_run *run, double *out, size_t capacity, size_t *n_written)
{
    if (pmf_status s = need_finished(run)) return s;
    if (run->items.size() != 1) return fail(PMF_EINVAL, "pmf_run_partials: single-item runs only");
    const size_t need = (size_t)kPartialDoubles * run->n_windows * run->replicas;
    if (n_written) *n_written = need;
    if (!out || capacity < need) return fail(PMF_EINVAL, "pmf_run_partials: capacity too small");
    const_cast<pmf_run *>(run)->reduced = false;  // the partials share the reduction scratch
    cudaError_t e = partials_launch(layout_of(run), run->d_scratch, g_stream);
    if (e != cudaSuccess) return cuda_fail(e, "partials");
    CK(cudaMemcpyAsync(out, run->d_scratch, sizeof(double) * need, cudaMemcpyDeviceToHost, g_stream), "copy");
    CK(cudaStreamSynchronize(g_stream), "sync");
    return PMF_OK;
}

// Eq. (5) / Eq. (15) on a filled reduction layout (device pointers); the
// caller's G, se_G (n_windows each) and dF_turn_on (one value), host.
static pmf_status state_common(const ReduceLayout &L, void *scratch, double *G, double *se_G, double *dF_turn_on)
{
    struct Tmp {
        void *pt = nullptr;
        double *out = nullptr;
        ~Tmp() { cudaFree(pt); cudaFree(out); }
    } t;
    const int s = L.n_windows;
    CK(cudaMalloc(&t.pt, partial_bytes(1, L.replicas)), "alloc turn-on partials");
    CK(cudaMalloc(&t.out, sizeof(double) * (2 * (size_t)s + 1)), "alloc state results");
    cudaError_t e = state_launch(L, scratch, t.pt, t.out, g_stream);
    if (e != cudaSuccess) return cuda_fail(e, "state free energy");
    std::vector<double> h(2 * (size_t)s + 1);
    CK(cudaMemcpyAsync(h.data(), t.out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, g_stream), "copy");
    CK(cudaStreamSynchronize(g_stream), "sync");
    if (G) std::memcpy(G, h.data(), sizeof(double) * s);
    if (se_G) std::memcpy(se_G, h.data() + s, sizeof(double) * s);
    if (dF_turn_on) *dF_turn_on = h[2 * (size_t)s];
    return PMF_OK;
}

pmf_status pmf_state_free_energy(pmf_run *run, double *G, double *se_G, double *dF_turn_on, int capacity)
{
    if (pmf_status s = need_finished(run)) return s;
    if (run->items.size() != 1 || run->d_w) return fail(PMF_EINVAL, "pmf_state_free_energy: single-path window runs only");
    if (capacity < run->n_windows) return fail(PMF_EINVAL, "pmf_state_free_energy: capacity smaller than n_windows");
    const ReduceLayout L = layout_of(run);
    cudaError_t e = reduce_launch(L, run->d_scratch, run->d_res, g_stream);
    if (e != cudaSuccess) return cuda_fail(e, "reduce");
    run->reduced = true;
    return state_common(L, run->d_scratch, G, se_G, dF_turn_on);
}

pmf_status pmf_state_free_energy_from_samples(const float *x, int x_on_device, const double *lambda, int n_windows,
                                              int replicas, const int64_t *samples_per_window, double k, double kT,
                                              double *G, double *se_G, double *dF_turn_on)
{
    if (!x || !lambda || !samples_per_window) return fail(PMF_EINVAL, "null argument");
    if (pmf_status s = need_device()) return s;
    if (n_windows < 1 || n_windows > 1024 || replicas < 1 || replicas > 65535)
        return fail(PMF_EINVAL, "bad window / replica count");
    if (!(k > 0) || !(kT > 0)) return fail(PMF_EINVAL, "need k > 0, kT > 0");
    std::vector<long long> off(n_windows), tw(n_windows);
    long long total = 0;
    for (int i = 0; i < n_windows; ++i) {
        if (samples_per_window[i] < 1) return fail(PMF_EINVAL, "each window needs at least one sample");
        tw[i] = samples_per_window[i];
        off[i] = total;
        total += tw[i] * replicas;
    }
    struct Tmp {
        double *lam = nullptr;
        long long *off = nullptr, *tw = nullptr;
        float *x = nullptr;
        void *scratch = nullptr;
        double *res = nullptr;
        ~Tmp() { cudaFree(lam); cudaFree(off); cudaFree(tw); cudaFree(x); cudaFree(scratch); cudaFree(res); }
    } t;
    CK(upload(&t.lam, lambda, n_windows), "upload lambda");
    CK(upload(&t.off, off.data(), n_windows), "upload offsets");
    CK(upload(&t.tw, tw.data(), n_windows), "upload counts");
    const float *dx = x;
    if (!x_on_device) {
        CK(upload(&t.x, x, (size_t)total), "upload samples");
        dx = t.x;
    }
    CK(cudaMalloc(&t.scratch, reduce_scratch_bytes(n_windows, replicas)), "alloc scratch");
    CK(cudaMalloc(&t.res, sizeof(double) * kResFields * n_windows), "alloc result");
    ReduceLayout L;
    L.x = dx;
    L.lambda = t.lam;
    L.off_w = t.off;
    L.tw = t.tw;
    L.n_windows = n_windows;
    L.replicas = replicas;
    L.k = k;
    L.kT = kT;
    cudaError_t e = reduce_launch(L, t.scratch, t.res, g_stream);
    if (e != cudaSuccess) return cuda_fail(e, "reduce");
    return state_common(L, t.scratch, G, se_G, dF_turn_on);
}

pmf_status pmf_free_energy_from_partials(const double *partials, const double *lambda, int n_windows, int replicas,
                                         double k, double kT, pmf_free_energy_result *res)
{
    if (!partials || !lambda || !res) return fail(PMF_EINVAL, "null argument");
    if (pmf_status s = need_device()) return s;
    if (n_windows < 2 || n_windows > kMaxRunWindows || replicas < 1 || replicas > (1 << 24))
        return fail(PMF_EINVAL, "bad window / replica count");
    if (res->capacity < n_windows) return fail(PMF_EINVAL, "result capacity smaller than n_windows");
    if (!(k > 0) || !(kT > 0)) return fail(PMF_EINVAL, "need k > 0, kT > 0");
    const size_t np = (size_t)kPartialDoubles * n_windows * replicas;
    for (size_t i = 0; i < np; i += kPartialDoubles)
        if (!(partials[i + 2] >= 0)) return fail(PMF_EINVAL, "partial sample counts must be >= 0");
    struct Tmp {
        double *lam = nullptr, *P = nullptr, *res = nullptr;
        void *wo = nullptr;
        ~Tmp() { cudaFree(lam); cudaFree(P); cudaFree(res); cudaFree(wo); }
    } t;
    CK(upload(&t.lam, lambda, n_windows), "upload lambda");
    CK(upload(&t.P, partials, np), "upload partials");
    CK(cudaMalloc(&t.wo, reduce_scratch_bytes(n_windows, replicas) - partial_bytes(n_windows, replicas)),
       "alloc scratch");
    CK(cudaMalloc(&t.res, sizeof(double) * kResFields * n_windows), "alloc results");
    ReduceLayout L;
    L.lambda = t.lam;
    L.n_windows = n_windows;
    L.replicas = replicas;
    L.k = k;
    L.kT = kT;
    cudaError_t e = combine_launch(L, t.P, t.wo, t.res, g_stream);
    if (e != cudaSuccess) return cuda_fail(e, "combine");
    std::vector<double> h((size_t)kResFields * n_windows);
    CK(cudaMemcpyAsync(h.data(), t.res, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, g_stream), "copy");
    CK(cudaStreamSynchronize(g_stream), "sync");
    return copy_result(h.data(), n_windows, res);
}

pmf_status pmf_free_energy_from_samples(const float *x, int x_on_device, const double *lambda, int n_windows,
                                        int replicas, const int64_t *samples_per_window, double k, double kT,
                                        pmf_free_energy_result *res)
{
    if (!x || !lambda || !samples_per_window || !res) return fail(PMF_EINVAL, "null argument");
    if (pmf_status s = need_device()) return s;
    if (n_windows < 2 || n_windows > 1024 || replicas < 1 || replicas > 65535)
        return fail(PMF_EINVAL, "bad window / replica count");
    if (res->capacity < n_windows) return fail(PMF_EINVAL, "result capacity smaller than n_windows");
    if (!(k > 0) || !(kT > 0)) return fail(PMF_EINVAL, "need k > 0, kT > 0");
    std::vector<long long> off(n_windows), tw(n_windows);
    long long total = 0;
    for (int i = 0; i < n_windows; ++i) {
        if (samples_per_window[i] < 1) return fail(PMF_EINVAL, "each window needs at least one sample");
        tw[i] = samples_per_window[i];
        off[i] = total;
        total += tw[i] * replicas;
    }
    struct Tmp {
        double *lam = nullptr, *res = nullptr;
        long long *off = nullptr, *tw = nullptr;
        float *x = nullptr;
        void *scratch = nullptr;
        ~Tmp() { cudaFree(lam); cudaFree(res); cudaFree(off); cudaFree(tw); cudaFree(x); cudaFree(scratch); }
    } t;
    CK(upload(&t.lam, lambda, n_windows), "upload lambda");
    CK(upload(&t.off, off.data(), n_windows), "upload offsets");
    CK(upload(&t.tw, tw.data(), n_windows), "upload counts");
    const float *dx = x;
    if (!x_on_device) {
        CK(upload(&t.x, x, (size_t)total), "upload samples");
        dx = t.x;
    }
    CK(cudaMalloc(&t.scratch, reduce_scratch_bytes(n_windows, replicas)), "alloc scratch");
    CK(cudaMalloc(&t.res, sizeof(double) * kResFields * n_windows), "alloc result");
    ReduceLayout L;
    L.x = dx;
    L.lambda = t.lam;
    L.off_w = t.off;
    L.tw = t.tw;
    L.n_windows = n_windows;
    L.replicas = replicas;
    L.k = k;
    L.kT = kT;
    cudaError_t e = reduce_launch(L, t.scratch, t.res, g_stream);
    if (e != cudaSuccess) return cuda_fail(e, "reduce");
    std::vector<double> h((size_t)kResFields * n_windows);
    CK(cudaMemcpyAsync(h.data(), t.res, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, g_stream), "copy");
    CK(cudaStreamSynchronize(g_stream), "sync");
    return copy_result(h.data(), n_windows, res);
}

// ---------------------------------------------------------------- surrogate MLP

struct pmf_mlp {
    float *params = nullptr, *m = nullptr, *v = nullptr;
    int *err = nullptr;
    int t = 0;
    double c = 0, h = 1;
    int split = 1;                   // training: one CTA per 128-sample tile
    float *tile_grad = nullptr;      // [tile_cap][kMlpParams]
    double *tile_loss = nullptr;     // [tile_cap]
    int tile_cap = 0;
    ~pmf_mlp()
    {
        cudaFree(params);
        cudaFree(m);
        cudaFree(v);
        cudaFree(err);
        cudaFree(tile_grad);
        cudaFree(tile_loss);
    }
};

pmf_status pmf_mlp_create(const float *params, double c, double h, pmf_mlp **out)
{
    if (!params || !out) return fail(PMF_EINVAL, "pmf_mlp_create: null argument");
    *out = nullptr;
    if (!std::isfinite(c) || !(h > 0) || !std::isfinite(h)) return fail(PMF_EINVAL, "pmf_mlp_create: need finite c, h > 0");
    for (int i = 0; i < kMlpParams; ++i)
        if (!std::isfinite(params[i])) return fail(PMF_EINVAL, "pmf_mlp_create: non-finite weight");
    if (pmf_status s = need_device()) return s;
    auto m = std::make_unique<pmf_mlp>();
    m->c = c;
    m->h = h;
    CK(upload(&m->params, params, kMlpParams), "mlp params");
    CK(cudaMalloc(&m->m, sizeof(float) * kMlpParams), "mlp adam");
    CK(cudaMalloc(&m->v, sizeof(float) * kMlpParams), "mlp adam");
    CK(cudaMemset(m->m, 0, sizeof(float) * kMlpParams), "mlp adam");
    CK(cudaMemset(m->v, 0, sizeof(float) * kMlpParams), "mlp adam");
    CK(cudaMalloc(&m->err, sizeof(int)), "mlp flag");
    CK(cudaMemset(m->err, 0, sizeof(int)), "mlp flag");
    *out = m.release();
    return PMF_OK;
}

void pmf_mlp_destroy(pmf_mlp *mlp) { delete mlp; }

pmf_status pmf_mlp_get_params(const pmf_mlp *mlp, float *params)
{
    if (!mlp || !params) return fail(PMF_EINVAL, "null argument");
    CK(cudaMemcpyAsync(params, mlp->params, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, g_stream), "copy");
    CK(cudaStreamSynchronize(g_stream), "sync");
    return PMF_OK;
}

static pmf_status mlp_run(pmf_mlp *mlp, MlpLaunch &L, const char *where)
{
    L.params = mlp->params;
    L.adam_m = mlp->m;
    L.adam_v = mlp->v;
    L.c = mlp->c;
    L.h = mlp->h;
    L.err = mlp->err;
    if (L.mode == 2 && mlp->split) {
        const int tiles = (L.batch + kMlpTile - 1) / kMlpTile;
        if (tiles > mlp->tile_cap) {
            cudaFree(mlp->tile_grad);
            cudaFree(mlp->tile_loss);
            mlp->tile_grad = nullptr;
            mlp->tile_loss = nullptr;
            mlp->tile_cap = 0;
            CK(cudaMalloc(&mlp->tile_grad, sizeof(float) * kMlpParams * tiles), where);
            CK(cudaMalloc(&mlp->tile_loss, sizeof(double) * tiles), where);
            mlp->tile_cap = tiles;
        }
        L.split = true;
        L.tile_grad = mlp->tile_grad;
        L.tile_loss = mlp->tile_loss;
        L.tile_cap = mlp->tile_cap;
    }
    CK(cudaMemsetAsync(mlp->err, 0, sizeof(int), g_stream), where);
    cudaError_t e = mlp_launch(L, g_stream);
    if (e != cudaSuccess) return cuda_fail(e, where);
    int err = 0;
    CK(cudaMemcpyAsync(&err, mlp->err, sizeof(int), cudaMemcpyDeviceToHost, g_stream), where);
    CK(cudaStreamSynchronize(g_stream), where);
    if (err) return fail(PMF_ETIMEOUT, std::string(where) + ": tensor-core completion wait timed out");
    return PMF_OK;
}

pmf_status pmf_mlp_predict(pmf_mlp *mlp, const double *lambda, int n, double *mu, double *log_var)
{
    if (!mlp || !lambda || !mu || !log_var || n < 0) return fail(PMF_EINVAL, "pmf_mlp_predict: bad argument");
    if (n == 0) return PMF_OK;
    struct Tmp {
        double *lam = nullptr, *mu = nullptr, *lv = nullptr;
        ~Tmp() { cudaFree(lam); cudaFree(mu); cudaFree(lv); }
    } t;
    CK(upload(&t.lam, lambda, n), "upload lambda");
    CK(cudaMalloc(&t.mu, sizeof(double) * n), "alloc");
    CK(cudaMalloc(&t.lv, sizeof(double) * n), "alloc");
    MlpLaunch L;
    L.mode = 0;
    L.lam_in = t.lam;
    L.n = n;
    L.out_mu = t.mu;
    L.out_logvar = t.lv;
    if (pmf_status s = mlp_run(mlp, L, "pmf_mlp_predict")) return s;
    CK(cudaMemcpy(mu, t.mu, sizeof(double) * n, cudaMemcpyDeviceToHost), "copy");
    CK(cudaMemcpy(log_var, t.lv, sizeof(double) * n, cudaMemcpyDeviceToHost), "copy");
    return PMF_OK;
}

pmf_status pmf_mlp_gradient(pmf_mlp *mlp, const double *lambda, const float *x, int n, float *grad, double *loss)
{
    if (!mlp || !lambda || !x || !grad || n < 1) return fail(PMF_EINVAL, "pmf_mlp_gradient: bad argument");
    struct Tmp {
        double *lam = nullptr, *loss = nullptr;
        float *x = nullptr, *g = nullptr;
        ~Tmp() { cudaFree(lam); cudaFree(loss); cudaFree(x); cudaFree(g); }
    } t;
    CK(upload(&t.lam, lambda, n), "upload lambda");
    CK(upload(&t.x, x, n), "upload x");
    CK(cudaMalloc(&t.g, sizeof(float) * kMlpParams), "alloc");
    CK(cudaMalloc(&t.loss, sizeof(double)), "alloc");
    MlpLaunch L;
    L.mode = 1;
    L.lam_in = t.lam;
    L.x_in = t.x;
    L.n = n;
    L.out_grad = t.g;
    L.out_loss = t.loss;
    if (pmf_status s = mlp_run(mlp, L, "pmf_mlp_gradient")) return s;
    CK(cudaMemcpy(grad, t.g, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost), "copy");
    if (loss) CK(cudaMemcpy(loss, t.loss, sizeof(double), cudaMemcpyDeviceToHost), "copy");
    return PMF_OK;
}

pmf_status pmf_mlp_set_split(pmf_mlp *mlp, int split)
{
    if (!mlp || (split != 0 && split != 1)) return fail(PMF_EINVAL, "pmf_mlp_set_split: bad argument");
    mlp->split = split;
    return PMF_OK;
}

pmf_status pmf_mlp_train(pmf_mlp *mlp, const pmf_run *run, int steps, int batch, double lr, uint64_t seed,
                         double *loss)
{
    if (!mlp || !run || steps < 0 || batch < 1 || batch > (1 << 20) || !(lr > 0))
        return fail(PMF_EINVAL, "pmf_mlp_train: bad argument");
    if (pmf_status s = need_finished(run)) return s;
    if (steps == 0) return PMF_OK;
    double *dloss = nullptr;
    CK(cudaMalloc(&dloss, sizeof(double)), "alloc");
    MlpLaunch L;
    L.mode = 2;
    L.adam_t = mlp->t;
    L.lr = lr;
    L.xs = run->d_x;
    L.win_lambda = run->d_lambda;
    L.win_off = run->d_off;
    L.win_tw = run->d_tw;
    L.n_windows = run->n_windows;
    L.replicas = run->replicas;
    L.total = run->total;
    L.steps = steps;
    L.batch = batch;
    L.seed = seed;
    L.out_loss = dloss;
    pmf_status s = mlp_run(mlp, L, "pmf_mlp_train");
    if (s == PMF_OK) {
        mlp->t += steps;
        if (loss) {
            cudaError_t e = cudaMemcpy(loss, dloss, sizeof(double), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) s = cuda_fail(e, "copy loss");
        }
    }
    cudaFree(dloss);
    return s;
}

// ---------------------------------------------------------------- adaptive protocol

namespace {


struct Window {
    double lam;
    pmf_run *run;
    int w;  // window index inside run
};

// Samples of several runs' windows merged in path order (device copies).
struct Merged {
    float *x = nullptr;
    double *lam = nullptr;
    long long *off = nullptr, *tw = nullptr;
    long long total = 0;
    int n = 0;
    ~Merged() { cudaFree(x); cudaFree(lam); cudaFree(off); cudaFree(tw); }
};

cudaError_t merge_windows(const std::vector<Window> &win, int replicas, Merged &m)
{
    m.n = (int)win.size();
    std::vector<double> lam(m.n);
    std::vector<long long> off(m.n), tw(m.n);
    long long total = 0;
    for (int i = 0; i < m.n; ++i) {
        lam[i] = win[i].lam;
        tw[i] = win[i].run->tw[win[i].w];
        off[i] = total;
        total += tw[i] * replicas;
    }
    m.total = total;
    cudaError_t e;
    if ((e = cudaMalloc(&m.x, sizeof(float) * total)) != cudaSuccess) return e;
    for (int i = 0; i < m.n; ++i) {
        const pmf_run *r = win[i].run;
        e = cudaMemcpyAsync(m.x + off[i], r->d_x + r->off[win[i].w], sizeof(float) * tw[i] * replicas,
                            cudaMemcpyDeviceToDevice, g_stream);
        if (e != cudaSuccess) return e;
    }
    if ((e = upload(&m.lam, lam.data(), m.n)) != cudaSuccess) return e;
    if ((e = upload(&m.off, off.data(), m.n)) != cudaSuccess) return e;
    return upload(&m.tw, tw.data(), m.n);
}

}  // namespace

pmf_status pmf_run_adaptive(pmf_system *sys, const double *lambda0, int n0, const pmf_run_params *p,
                            const pmf_adaptive_params *ap, pmf_adaptive_info *info, pmf_free_energy_result *res)
{
    if (!sys || !lambda0 || !p || !ap || !info || !res || !ap->mlp_init)
        return fail(PMF_EINVAL, "pmf_run_adaptive: null argument");
    if (ap->max_windows < n0 || ap->max_windows > 1024 || ap->max_rounds < 0 || !(ap->overlap_threshold >= 0) ||
        ap->overlap_threshold > 1 || ap->mlp_steps < 0 || ap->mlp_batch < 1 || !(ap->mlp_lr > 0))
        return fail(PMF_EINVAL, "pmf_run_adaptive: bad adaptive parameters");
    if (res->capacity < ap->max_windows) return fail(PMF_EINVAL, "pmf_run_adaptive: result capacity < max_windows");
    pmf_adaptive_trace *tr = ap->trace;
    if (tr) {
        if (tr->max_rounds < 0 || tr->max_windows < ap->max_windows || tr->replicas != p->replicas ||
            p->replicas > kMaxSeedCandidates / 2)
            return fail(PMF_EINVAL, "pmf_run_adaptive: trace needs max_windows >= the protocol's, "
                                    "replicas = the run's (<= 2048)");
        tr->rounds = 0;
    }
    std::memset(info, 0, sizeof(*info));
    GpuTimer timer;
    // Launches with few replicas per SM run faster with more warps per
    // replica (more resident warps to hide latency): unless the caller chose
    // the chain's warp count, each launch of an FP32 chain takes 8 warps
    // below three replicas per SM and 4 otherwise; the default is restored
    // on return.
    struct WarpScope {
        ChainModel *m = nullptr;
        bool changed = false;
        ~WarpScope()
        {
            if (m && changed) m->set_warps(4);
        }
    } wscope;
    int sms = 1;
    {
        int dev = 0;
        CK(cudaGetDevice(&dev), "pmf_run_adaptive");
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "pmf_run_adaptive");
    }
    if (sys->model == PMF_MODEL_CHAIN && sys->chains[p->chain]->precision() != PMF_FP64 &&
        sys->chains[p->chain]->warps() == 4 &&
        !(p->chain < (int)sys->warps_chosen.size() && sys->warps_chosen[p->chain]))
        wscope.m = sys->chains[p->chain].get();
    auto pick_warps = [&](long long n_rep) -> pmf_status {
        if (!wscope.m) return PMF_OK;
        const int nw = n_rep < 3LL * sms ? 8 : 4;
        if (wscope.m->warps() == nw) return PMF_OK;
        wscope.changed = true;
        cudaError_t e = wscope.m->set_warps(nw);
        if (e == cudaSuccess && wscope.m->smem_bytes() > 227 * 1024 - 256) e = wscope.m->set_warps(4);
        return e == cudaSuccess ? PMF_OK : cuda_fail(e, "pmf_run_adaptive: warps");
    };
    std::vector<std::unique_ptr<pmf_run, void (*)(pmf_run *)>> runs;
    auto own = [&](pmf_run *r) { runs.emplace_back(r, pmf_destroy_run); };
    pmf_run *r0 = nullptr;
    pmf_status st = pmf_run_prepare(sys, lambda0, n0, p, &r0);
    if (st != PMF_OK) return st;
    own(r0);
    if ((st = pick_warps((long long)n0 * p->replicas)) != PMF_OK) return st;
    timer.start();
    if ((st = pmf_run_launch(r0)) != PMF_OK) return st;
    if ((st = pmf_run_wait(r0)) != PMF_OK) return st;
    CK(timer.stop(), "timer");
    const double dir = lambda0[n0 - 1] > lambda0[0] ? 1.0 : -1.0;
    std::vector<Window> win;
    for (int i = 0; i < n0; ++i) win.push_back(Window{lambda0[i], r0, i});
    uint32_t uid_next = p->uid_base + (uint32_t)(n0 * p->replicas);
    const int R = p->replicas;
    double lo = lambda0[0], hi = lambda0[0];
    for (int i = 0; i < n0; ++i) { lo = std::min(lo, lambda0[i]); hi = std::max(hi, lambda0[i]); }
    pmf_mlp *mlp_raw = nullptr;
    if ((st = pmf_mlp_create(ap->mlp_init, 0.5 * (lo + hi), std::max(0.5 * (hi - lo), 1e-6), &mlp_raw)) != PMF_OK)
        return st;
    std::unique_ptr<pmf_mlp, void (*)(pmf_mlp *)> mlp(mlp_raw, pmf_mlp_destroy);
    const bool chain = sys->model == PMF_MODEL_CHAIN;
    const int N = chain ? sys->chains[p->chain]->n_beads() : 0;
    const int Np = chain ? sys->chains[p->chain]->n_padded() : 0;
    const bool fp64 = chain && sys->chains[p->chain]->precision() == PMF_FP64;
    const size_t state_stride = chain ? sys->chains[p->chain]->state_bytes_per_replica() : 2 * sizeof(double);
    for (int round = 0; round < ap->max_rounds; ++round) {
        std::sort(win.begin(), win.end(), [&](const Window &a, const Window &b) { return dir * a.lam < dir * b.lam; });
        Merged m;
        timer.start();
        CK(merge_windows(win, R, m), "merge samples");
        const bool rec = tr && round < tr->max_rounds;
        if (ap->train_on_gap) {
            // the measured moments first: without a gap between neighbours no
            // window would be inserted, so the round ends the protocol untrained
            std::vector<double> dovl(m.n > 1 ? m.n - 1 : 0);
            double *d_mu = nullptr, *d_lv = nullptr, *d_ovl = nullptr;
            cudaError_t e = cudaMalloc(&d_mu, sizeof(double) * m.n);
            if (e == cudaSuccess) e = cudaMalloc(&d_lv, sizeof(double) * m.n);
            if (e == cudaSuccess) e = cudaMalloc(&d_ovl, sizeof(double) * std::max<size_t>(1, dovl.size()));
            if (e == cudaSuccess) e = moments_launch(m.x, m.off, m.tw, R, m.n, d_mu, d_lv, g_stream);
            if (e == cudaSuccess) e = overlap_launch(d_mu, d_lv, m.n, d_ovl, g_stream);
            if (e == cudaSuccess && !dovl.empty())
                e = cudaMemcpyAsync(dovl.data(), d_ovl, sizeof(double) * dovl.size(), cudaMemcpyDeviceToHost, g_stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
            cudaFree(d_mu);
            cudaFree(d_lv);
            cudaFree(d_ovl);
            if (e != cudaSuccess) return cuda_fail(e, "measured overlap");
            bool gap = false;
            for (double v : dovl) gap = gap || v < ap->overlap_threshold;
            if (rec) {
                const size_t o = (size_t)round * tr->max_windows;
                if (tr->data_ovl)
                    for (size_t i = 0; i < dovl.size(); ++i) tr->data_ovl[o + i] = dovl[i];
                if (tr->trained) tr->trained[round] = gap ? 1 : 0;
            }
            if (!gap) {
                CK(timer.stop(), "timer");
                if (rec) {
                    const size_t o = (size_t)round * tr->max_windows;
                    if (tr->n_windows) tr->n_windows[round] = m.n;
                    if (tr->n_inserted) tr->n_inserted[round] = 0;
                    for (int i = 0; i < m.n; ++i) {
                        if (tr->lambda) tr->lambda[o + i] = win[i].lam;
                        if (tr->mu) tr->mu[o + i] = NAN;
                        if (tr->log_var) tr->log_var[o + i] = NAN;
                        if (tr->ovl && i + 1 < m.n) tr->ovl[o + i] = NAN;
                    }
                    tr->rounds = round + 1;
                }
                break;
            }
        } else if (rec && tr->trained) {
            tr->trained[round] = 1;
        }
        MlpLaunch L;
        L.mode = 2;
        L.adam_t = mlp->t;
        L.lr = ap->mlp_lr;
        L.xs = m.x;
        L.win_lambda = m.lam;
        L.win_off = m.off;
        L.win_tw = m.tw;
        L.n_windows = m.n;
        L.replicas = R;
        L.total = m.total;
        L.steps = ap->mlp_steps;
        L.batch = ap->mlp_batch;
        L.seed = ap->mlp_seed + (uint64_t)round;
        double *dloss = nullptr;
        CK(cudaMalloc(&dloss, sizeof(double)), "alloc");
        L.out_loss = dloss;
        if (ap->mlp_steps > 0) {
            if ((st = mlp_run(mlp.get(), L, "pmf_run_adaptive: training")) != PMF_OK) { cudaFree(dloss); return st; }
            mlp->t += ap->mlp_steps;
            cudaMemcpy(&info->mlp_loss, dloss, sizeof(double), cudaMemcpyDeviceToHost);
        }
        cudaFree(dloss);
        // predictions at the windows and at the candidate midpoints
        std::vector<double> lam(m.n), mids(m.n > 1 ? m.n - 1 : 0);
        for (int i = 0; i < m.n; ++i) lam[i] = win[i].lam;
        for (int i = 0; i + 1 < m.n; ++i) mids[i] = 0.5 * (lam[i] + lam[i + 1]);
        std::vector<double> mu(m.n), lv(m.n), mu_mid(mids.size()), lv_mid(mids.size()), ovl(mids.size());
        if ((st = pmf_mlp_predict(mlp.get(), lam.data(), m.n, mu.data(), lv.data())) != PMF_OK) return st;
        if (!mids.empty() && (st = pmf_mlp_predict(mlp.get(), mids.data(), (int)mids.size(), mu_mid.data(), lv_mid.data())) != PMF_OK)
            return st;
        {
            double *d_mu = nullptr, *d_lv = nullptr, *d_ovl = nullptr;
            cudaError_t e = upload(&d_mu, mu.data(), m.n);
            if (e == cudaSuccess) e = upload(&d_lv, lv.data(), m.n);
            if (e == cudaSuccess) e = cudaMalloc(&d_ovl, sizeof(double) * std::max<size_t>(1, mids.size()));
            if (e == cudaSuccess) e = overlap_launch(d_mu, d_lv, m.n, d_ovl, g_stream);
            if (e == cudaSuccess && !mids.empty())
                e = cudaMemcpyAsync(ovl.data(), d_ovl, sizeof(double) * mids.size(), cudaMemcpyDeviceToHost, g_stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
            cudaFree(d_mu);
            cudaFree(d_lv);
            cudaFree(d_ovl);
            if (e != cudaSuccess) return cuda_fail(e, "overlap");
        }
        CK(timer.stop(), "timer");
        std::vector<int> pick;
        for (size_t i = 0; i < mids.size(); ++i)
            if (ovl[i] < ap->overlap_threshold && (int)(win.size() + pick.size()) < ap->max_windows) pick.push_back((int)i);
        if (rec) {
            const size_t o = (size_t)round * tr->max_windows;
            if (tr->n_windows) tr->n_windows[round] = m.n;
            if (tr->n_inserted) tr->n_inserted[round] = (int)pick.size();
            for (int i = 0; i < m.n; ++i) {
                if (tr->lambda) tr->lambda[o + i] = lam[i];
                if (tr->mu) tr->mu[o + i] = mu[i];
                if (tr->log_var) tr->log_var[o + i] = lv[i];
                if (tr->ovl && i + 1 < m.n) tr->ovl[o + i] = ovl[i];
            }
            for (size_t q = 0; q < pick.size(); ++q) {
                if (tr->inserted) tr->inserted[o + q] = mids[pick[q]];
                if (tr->target) tr->target[o + q] = mu_mid[pick[q]];
            }
            tr->rounds = round + 1;
        }
        if (pick.empty()) break;
        // the next launch: the inserted windows, seeded from the end states of
        // their two neighbours, and (with continuation) every current window,
        // continued from its own replicas' end states, all in one run
        struct Next {
            double lam;
            int inserted;  // 1: midpoint pick[idx]; 0: current window win[idx]
            int idx;
        };
        std::vector<Next> next;
        for (size_t q = 0; q < pick.size(); ++q) next.push_back(Next{mids[pick[q]], 1, (int)q});
        if (ap->continue_windows)
            for (size_t i = 0; i < win.size(); ++i) next.push_back(Next{win[i].lam, 0, (int)i});
        std::sort(next.begin(), next.end(), [&](const Next &a, const Next &b) { return dir * a.lam < dir * b.lam; });
        std::vector<SeedJob> jobs(next.size());
        std::vector<double> new_lam(next.size());
        std::vector<int> job_of_pick(pick.size(), 0);
        int max_cand = 0;
        for (size_t j = 0; j < next.size(); ++j) {
            new_lam[j] = next[j].lam;
            int nc = 0;
            if (next[j].inserted) {
                const int i = pick[next[j].idx];
                job_of_pick[next[j].idx] = (int)j;
                jobs[j].target = mu_mid[i];
                for (int side = 0; side < 2; ++side) {
                    const Window &nb = win[i + side];
                    for (int r = 0; r < R && nc < kMaxSeedCandidates; ++r) {
                        const size_t rep = (size_t)nb.w * nb.run->replicas + r;
                        jobs[j].cand[nc++] = static_cast<const char *>(nb.run->d_state) + rep * state_stride;
                    }
                }
            } else {
                // continuation: replica r resumes from replica r's end state
                // (a NaN target keeps the candidates in order)
                const Window &cw = win[next[j].idx];
                jobs[j].target = NAN;
                for (int r = 0; r < R && nc < kMaxSeedCandidates; ++r) {
                    const size_t rep = (size_t)cw.w * cw.run->replicas + r;
                    jobs[j].cand[nc++] = static_cast<const char *>(cw.run->d_state) + rep * state_stride;
                }
            }
            jobs[j].n_cand = nc;
            max_cand = std::max(max_cand, nc);
        }
        pmf_run_params p2 = *p;
        p2.uid_base = uid_next;
        p2.n_steps_per_window = nullptr;
        pmf_run *rn = nullptr;
        if ((st = pmf_run_prepare(sys, new_lam.data(), (int)new_lam.size(), &p2, &rn)) != PMF_OK) return st;
        own(rn);
        SeedJob *d_jobs = nullptr;
        timer.start();
        CK(upload(&d_jobs, jobs.data(), jobs.size()), "upload seed jobs");
        const size_t per = chain ? 3 * (size_t)N : 1;
        cudaError_t e = cudaMalloc(&rn->d_start, sizeof(double) * per * R * new_lam.size());
        int *d_choice = nullptr;
        double *d_cx = nullptr;
        if (rec && e == cudaSuccess && (tr->seed || tr->cand_x)) {
            e = cudaMalloc(&d_choice, sizeof(int) * R * jobs.size());
            if (e == cudaSuccess) e = cudaMalloc(&d_cx, sizeof(double) * max_cand * jobs.size());
        }
        if (e == cudaSuccess)
            e = seed_launch(d_jobs, (int)jobs.size(), max_cand, N, Np, R, fp64, rn->d_start, d_choice, d_cx, g_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
        if (e == cudaSuccess && d_choice) {
            std::vector<int> hc((size_t)R * jobs.size());
            std::vector<double> hx((size_t)max_cand * jobs.size());
            e = cudaMemcpy(hc.data(), d_choice, sizeof(int) * hc.size(), cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemcpy(hx.data(), d_cx, sizeof(double) * hx.size(), cudaMemcpyDeviceToHost);
            const size_t o = (size_t)round * tr->max_windows;
            for (size_t q = 0; e == cudaSuccess && q < pick.size(); ++q) {
                const size_t j = (size_t)job_of_pick[q];
                for (int r = 0; r < R && tr->seed; ++r) tr->seed[(o + q) * R + r] = hc[j * R + r];
                for (int c = 0; c < 2 * R && tr->cand_x; ++c)
                    tr->cand_x[(o + q) * 2 * R + c] = c < jobs[j].n_cand ? hx[j * max_cand + c] : NAN;
            }
        }
        cudaFree(d_choice);
        cudaFree(d_cx);
        cudaFree(d_jobs);
        if (e != cudaSuccess) return cuda_fail(e, "seed");
        if ((st = pick_warps((long long)new_lam.size() * R)) != PMF_OK) return st;
        if ((st = pmf_run_launch(rn)) != PMF_OK) return st;
        if ((st = pmf_run_wait(rn)) != PMF_OK) return st;
        CK(timer.stop(), "timer");
        if (ap->continue_windows) win.clear();  // every window's latest samples are in rn
        for (size_t q = 0; q < new_lam.size(); ++q) win.push_back(Window{new_lam[q], rn, (int)q});
        uid_next += (uint32_t)(new_lam.size() * R);
        info->rounds = round + 1;
        info->inserted += (int)pick.size();
    }
    std::sort(win.begin(), win.end(), [&](const Window &a, const Window &b) { return dir * a.lam < dir * b.lam; });
    Merged m;
    timer.start();
    CK(merge_windows(win, R, m), "merge samples");
    void *scratch = nullptr;
    double *d_res = nullptr;
    CK(cudaMalloc(&scratch, reduce_scratch_bytes(m.n, R)), "alloc");
    cudaError_t e = cudaMalloc(&d_res, sizeof(double) * kResFields * m.n);
    ReduceLayout RL;
    RL.x = m.x;
    RL.lambda = m.lam;
    RL.off_w = m.off;
    RL.tw = m.tw;
    RL.n_windows = m.n;
    RL.replicas = R;
    RL.k = p->k;
    RL.kT = p->kT;
    if (e == cudaSuccess) e = reduce_launch(RL, scratch, d_res, g_stream);
    std::vector<double> h((size_t)kResFields * m.n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d_res, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, g_stream);
    if (e == cudaSuccess) e = timer.stop();
    cudaFree(scratch);
    cudaFree(d_res);
    if (e != cudaSuccess) return cuda_fail(e, "reduce");
    info->n_windows = m.n;
    for (int i = 0; i < m.n; ++i) info->lambda[i] = win[i].lam;
    info->gpu_seconds = timer.ms / 1000.0;
    return copy_result(h.data(), m.n, res);
}

pmf_status pmf_chain_set_warps(pmf_system *sys, int chain, int warps)
{
    if (!sys || sys->model != PMF_MODEL_CHAIN || chain < 0 || chain >= (int)sys->chains.size())
        return fail(PMF_EINVAL, "pmf_chain_set_warps: not a chain system / bad chain index");
    cudaError_t e = sys->chains[chain]->set_warps(warps);
    if (e == cudaErrorInvalidValue) return fail(PMF_EINVAL, "pmf_chain_set_warps: warps must be 4, 5, 6 or 8 (FP64: 4)");
    if (e != cudaSuccess) return cuda_fail(e, "pmf_chain_set_warps");
    if (sys->chains[chain]->smem_bytes() > 227 * 1024 - 256) {
        sys->chains[chain]->set_warps(4);
        return fail(PMF_EINVAL, "pmf_chain_set_warps: shared memory would exceed 227 KB");
    }
    if (sys->warps_chosen.size() < sys->chains.size()) sys->warps_chosen.resize(sys->chains.size(), 0);
    sys->warps_chosen[chain] = 1;
    return PMF_OK;
}

pmf_status pmf_chain_set_grid(pmf_system *sys, int chain, int ctas, int seg_steps)
{
    if (!sys || sys->model != PMF_MODEL_CHAIN || chain < 0 || chain >= (int)sys->chains.size())
        return fail(PMF_EINVAL, "pmf_chain_set_grid: not a chain system / bad chain index");
    if (seg_steps < 0) return fail(PMF_EINVAL, "pmf_chain_set_grid: seg_steps must be >= 0");
    cudaError_t e = sys->chains[chain]->set_grid(ctas, seg_steps);
    if (e != cudaSuccess) return cuda_fail(e, "pmf_chain_set_grid");
    return PMF_OK;
}

pmf_status pmf_chain_set_schedule(pmf_system *sys, int chain, int variant)
{
    if (!sys || sys->model != PMF_MODEL_CHAIN || chain < 0 || chain >= (int)sys->chains.size())
        return fail(PMF_EINVAL, "pmf_chain_set_schedule: not a chain system / bad chain index");
    cudaError_t e = sys->chains[chain]->set_schedule_variant(variant);
    if (e == cudaErrorInvalidValue) return fail(PMF_EINVAL, "pmf_chain_set_schedule: variant out of range");
    if (e != cudaSuccess) return cuda_fail(e, "pmf_chain_set_schedule");
    return PMF_OK;
}

pmf_status pmf_chain_get_schedule(const pmf_system *sys, int chain, int *variant)
{
    if (!sys || sys->model != PMF_MODEL_CHAIN || chain < 0 || chain >= (int)sys->chains.size() || !variant)
        return fail(PMF_EINVAL, "pmf_chain_get_schedule: not a chain system / bad chain index / null output");
    *variant = sys->chains[chain]->schedule_variant();
    return PMF_OK;
}

pmf_status pmf_chain_get_launch(const pmf_system *sys, int chain, int *warps, int *ctas, int *seg_steps)
{
    if (!sys || sys->model != PMF_MODEL_CHAIN || chain < 0 || chain >= (int)sys->chains.size())
        return fail(PMF_EINVAL, "pmf_chain_get_launch: not a chain system / bad chain index");
    const ChainModel &m = *sys->chains[chain];
    if (warps) *warps = m.warps();
    if (ctas) *ctas = m.grid_ctas();
    if (seg_steps) *seg_steps = m.seg_steps();
    return PMF_OK;
}

pmf_status pmf_fp32_peak(int packed, int ctas_per_sm, int iters, int reps, double *tflops, double *ms)
{
    if (iters < 1 || reps < 1 || ctas_per_sm < 0 || ctas_per_sm > 64)
        return fail(PMF_EINVAL, "pmf_fp32_peak: iters >= 1, reps >= 1, 0 <= ctas_per_sm <= 64");
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev), "pmf_fp32_peak");
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "pmf_fp32_peak");
    const int ctas = (ctas_per_sm > 0 ? ctas_per_sm : 4) * sms;
    float *out = nullptr;
    CK(cudaMalloc(&out, sizeof(float) * (size_t)ctas * fp32_peak_threads()), "pmf_fp32_peak alloc");
    std::unique_ptr<float, cudaError_t (*)(void *)> guard(out, cudaFree);
    double flops = 0.0;
    CK(fp32_peak_launch(packed != 0, ctas, iters, out, &flops, g_stream), "pmf_fp32_peak warm-up");
    double best = 1e300;
    for (int r = 0; r < reps; ++r) {
        GpuTimer timer;
        timer.start();
        CK(fp32_peak_launch(packed != 0, ctas, iters, out, &flops, g_stream), "pmf_fp32_peak launch");
        CK(timer.stop(), "pmf_fp32_peak timer");
        best = std::min(best, timer.ms);
    }
    if (tflops) *tflops = flops / (best * 1e-3) / 1e12;
    if (ms) *ms = best;
    return PMF_OK;
}

pmf_status pmf_fp64_peak(int ctas_per_sm, int iters, int reps, double *tflops, double *ms)
{
    if (iters < 1 || reps < 1 || ctas_per_sm < 0 || ctas_per_sm > 64)
        return fail(PMF_EINVAL, "pmf_fp64_peak: iters >= 1, reps >= 1, 0 <= ctas_per_sm <= 64");
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev), "pmf_fp64_peak");
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "pmf_fp64_peak");
    const int ctas = (ctas_per_sm > 0 ? ctas_per_sm : 4) * sms;
    double *out = nullptr;
    CK(cudaMalloc(&out, sizeof(double) * (size_t)ctas * fp32_peak_threads()), "pmf_fp64_peak alloc");
    std::unique_ptr<double, cudaError_t (*)(void *)> guard(out, cudaFree);
    double flops = 0.0;
    CK(fp64_peak_launch(ctas, iters, out, &flops, g_stream), "pmf_fp64_peak warm-up");
    double best = 1e300;
    for (int r = 0; r < reps; ++r) {
        GpuTimer timer;
        timer.start();
        CK(fp64_peak_launch(ctas, iters, out, &flops, g_stream), "pmf_fp64_peak launch");
        CK(timer.stop(), "pmf_fp64_peak timer");
        best = std::min(best, timer.ms);
    }
    if (tflops) *tflops = flops / (best * 1e-3) / 1e12;
    if (ms) *ms = best;
    return PMF_OK;
}

pmf_status pmf_chain_autotune(pmf_system *sys, const double *lambda, int n_windows, const pmf_run_params *p,
                              int probe_steps, int *best_warps, double *best_ms)
{
    if (!sys || !lambda || !p || probe_steps < 1) return fail(PMF_EINVAL, "pmf_chain_autotune: bad argument");
    if (sys->model != PMF_MODEL_CHAIN) return fail(PMF_EINVAL, "pmf_chain_autotune: not a chain system");
    ChainModel &m = *sys->chains[p->chain];
    const int cand_fp32[4] = {4, 5, 6, 8};
    const int n_cand = m.precision() == PMF_FP64 ? 1 : 4;
    pmf_run_params q = *p;
    q.n_steps = probe_steps + 1;
    q.n_steps_per_window = nullptr;
    q.n_equil = probe_steps;
    q.sample_stride = 1;
    q.timeout_s = 0;
    pmf_run *run = nullptr;
    if (pmf_status s = pmf_run_prepare(sys, lambda, n_windows, &q, &run)) return s;
    std::unique_ptr<pmf_run, void (*)(pmf_run *)> guard(run, pmf_destroy_run);
    int best = m.warps(), best_grid = m.grid_ctas();
    const int seg = m.seg_steps();
    double best_t = 1e300;
    GpuTimer timer;
    // launch shapes: the automatic persistent grid, and one persistent CTA
    // per replica (equal to auto when the replicas fill every CTA slot)
    const int n_rep = n_windows * p->replicas;
    const int grids[2] = {0, n_rep};
    for (int c = 0; c < n_cand; ++c) {
        if (pmf_chain_set_warps(sys, p->chain, cand_fp32[c]) != PMF_OK) continue;
        for (int gsel = 0; gsel < 2; ++gsel) {
            if (m.set_grid(grids[gsel], seg) != cudaSuccess) continue;
            if (pmf_status s = pmf_run_launch(run)) return s;  // warm-up (and graph capture)
            if (pmf_status s = pmf_run_wait(run)) return s;
            double t = 1e300;
            for (int rep = 0; rep < 2; ++rep) {  // best of two timed launches
                const double before = timer.ms;
                timer.start();
                if (pmf_status s = pmf_run_launch(run)) return s;
                CK(timer.stop(), "autotune timer");
                if (pmf_status s = pmf_run_wait(run)) return s;
                t = std::min(t, timer.ms - before);
            }
            if (t < best_t) {
                best_t = t;
                best = cand_fp32[c];
                best_grid = grids[gsel];
            }
        }
    }
    if (pmf_status s = pmf_chain_set_warps(sys, p->chain, best)) return s;
    if (m.set_grid(best_grid, seg) != cudaSuccess) return fail(PMF_EINVAL, "pmf_chain_autotune: grid");
    // then the cost models of the FP32 schedule for that shape: each one
    // that gives a schedule not timed yet is probed the same way
    int best_v = m.schedule_variant();
    if (m.precision() != PMF_FP64) {
        std::vector<std::vector<std::vector<UnitDesc>>> seen;
        auto key = [&](int v) { return chain_schedule(m.n_beads(), best, true, v); };
        auto same = [](const std::vector<std::vector<UnitDesc>> &a, const std::vector<std::vector<UnitDesc>> &b) {
            if (a.size() != b.size()) return false;
            for (size_t w = 0; w < a.size(); ++w) {
                if (a[w].size() != b[w].size()) return false;
                for (size_t q = 0; q < a[w].size(); ++q)
                    if (std::memcmp(&a[w][q], &b[w][q], sizeof(UnitDesc)) != 0) return false;
            }
            return true;
        };
        seen.push_back(key(best_v));  // timed above
        for (int v = 0; v < kSchedVariants; ++v) {
            const auto sv = key(v);
            bool dup = false;
            for (const auto &o : seen) dup = dup || same(o, sv);
            if (dup) continue;
            seen.push_back(sv);
            if (m.set_schedule_variant(v) != cudaSuccess) continue;
            if (pmf_status s = pmf_run_launch(run)) return s;
            if (pmf_status s = pmf_run_wait(run)) return s;
            double t = 1e300;
            for (int rep = 0; rep < 2; ++rep) {
                const double before = timer.ms;
                timer.start();
                if (pmf_status s = pmf_run_launch(run)) return s;
                CK(timer.stop(), "autotune timer");
                if (pmf_status s = pmf_run_wait(run)) return s;
                t = std::min(t, timer.ms - before);
            }
            if (t < best_t) {
                best_t = t;
                best_v = v;
            }
        }
        if (m.set_schedule_variant(best_v) != cudaSuccess) return fail(PMF_EINVAL, "pmf_chain_autotune: schedule");
    }
    if (best_warps) *best_warps = best;
    if (best_ms) *best_ms = best_t;
    return PMF_OK;
}

pmf_status pmf_overlap(const double *mu, const double *log_var, int n, double *ovl)
{
    if (!mu || !log_var || !ovl || n < 2) return fail(PMF_EINVAL, "pmf_overlap: bad argument");
    if (pmf_status s = need_device()) return s;
    double *d_mu = nullptr, *d_lv = nullptr, *d_ovl = nullptr;
    cudaError_t e = upload(&d_mu, mu, n);
    if (e == cudaSuccess) e = upload(&d_lv, log_var, n);
    if (e == cudaSuccess) e = cudaMalloc(&d_ovl, sizeof(double) * (n - 1));
    if (e == cudaSuccess) e = overlap_launch(d_mu, d_lv, n, d_ovl, g_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ovl, d_ovl, sizeof(double) * (n - 1), cudaMemcpyDeviceToHost, g_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
    cudaFree(d_mu);
    cudaFree(d_lv);
    cudaFree(d_ovl);
    if (e != cudaSuccess) return cuda_fail(e, "pmf_overlap");
    return PMF_OK;
}

pmf_status pmf_free_energy_noalloc(const float *x, const double *lambda, int n_windows, int replicas,
                                   int64_t samples_per_window, double k, double kT, double *out)
{
    if (!x || !lambda || !out) return fail(PMF_EINVAL, "pmf_free_energy_noalloc: null pointer");
    if (n_windows < 2 || n_windows > kNoAllocMaxWindows)
        return fail(PMF_EINVAL, "pmf_free_energy_noalloc: n_windows must be in [2, 1024]");
    if (replicas < 1 || (long long)n_windows * replicas > kNoAllocMaxWindowReplicas)
        return fail(PMF_EINVAL, "pmf_free_energy_noalloc: n_windows * replicas must be in [1, 65536] "
                                "(fixed scratch size)");
    if (samples_per_window < 1) return fail(PMF_EINVAL, "pmf_free_energy_noalloc: samples_per_window >= 1");
    if (!(k > 0) || !(kT > 0)) return fail(PMF_EINVAL, "pmf_free_energy_noalloc: need k > 0, kT > 0");
    cudaError_t e = reduce_noalloc_launch(x, lambda, n_windows, replicas, samples_per_window, k, kT, out, g_stream);
    if (e != cudaSuccess) return cuda_fail(e, "pmf_free_energy_noalloc");
    return PMF_OK;
}

pmf_status pmf_final_state(const pmf_run *run, double *pos, double *vel, size_t capacity, size_t *n_written)
{
    if (pmf_status s = need_finished(run)) return s;
    const int n_rep = (run->sequential ? 1 : run->n_windows) * run->replicas;
    if (run->sys->model == PMF_MODEL_1D_DOUBLEWELL) {
        if (n_written) *n_written = (size_t)n_rep;
        if (!pos || capacity < (size_t)n_rep) return fail(PMF_EINVAL, "pmf_final_state: capacity too small");
        std::vector<double> st(2 * (size_t)n_rep);  // (x, pulling work) per simulation
        CK(cudaMemcpy(st.data(), run->d_state, sizeof(double) * st.size(), cudaMemcpyDeviceToHost), "copy state");
        for (int q = 0; q < n_rep; ++q) pos[q] = st[2 * (size_t)q];
        return PMF_OK;
    }
    size_t need = 0;
    const auto sims = [&](const RunItem &ri) { return (run->sequential ? 1 : ri.nw) * run->replicas; };
    for (const RunItem &ri : run->items) need += (size_t)sims(ri) * run->sys->chains[ri.chain]->n_beads() * 3;
    if (n_written) *n_written = need;
    if ((!pos && !vel) || capacity < need) return fail(PMF_EINVAL, "pmf_final_state: capacity too small");
    std::vector<unsigned char> raw(run->state_bytes);
    CK(cudaMemcpy(raw.data(), run->d_state, run->state_bytes, cudaMemcpyDeviceToHost), "copy state");
    size_t o = 0;
    for (const RunItem &ri : run->items) {
        const ChainModel &m = *run->sys->chains[ri.chain];
        const int N = m.n_beads(), Np = m.n_padded();
        const bool dbl = m.precision() == PMF_FP64;
        const unsigned char *base = raw.data() + ri.state_off;
        for (int q = 0; q < sims(ri); ++q)
            for (int b = 0; b < N; ++b, o += 3)
                for (int a = 0; a < 3; ++a) {
                    const size_t ip = ((size_t)q * 2 * Np + b) * 4 + a, iv = ((size_t)q * 2 * Np + Np + b) * 4 + a;
                    const double pv = dbl ? reinterpret_cast<const double *>(base)[ip] : reinterpret_cast<const float *>(base)[ip];
                    const double vv = dbl ? reinterpret_cast<const double *>(base)[iv] : reinterpret_cast<const float *>(base)[iv];
                    if (pos) pos[o + a] = pv;
                    if (vel) vel[o + a] = vv;
                }
    }
    return PMF_OK;
}

pmf_status pmf_philox(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int n_blocks, uint32_t *raw,
                      float *normals)
{
    if (n_blocks < 0) return fail(PMF_EINVAL, "n_blocks < 0");
    if (pmf_status s = need_device()) return s;
    if (n_blocks == 0) return PMF_OK;
    uint32_t *dr = nullptr;
    float *dn = nullptr;
    CK(cudaMalloc(&dr, sizeof(uint32_t) * 4 * n_blocks), "alloc");
    cudaError_t e = cudaMalloc(&dn, sizeof(float) * 4 * n_blocks);
    if (e == cudaSuccess) e = philox_launch(seed, c0, c1, c2, c3, n_blocks, dr, dn, g_stream);
    if (e == cudaSuccess && raw) e = cudaMemcpyAsync(raw, dr, sizeof(uint32_t) * 4 * n_blocks, cudaMemcpyDeviceToHost, g_stream);
    if (e == cudaSuccess && normals) e = cudaMemcpyAsync(normals, dn, sizeof(float) * 4 * n_blocks, cudaMemcpyDeviceToHost, g_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
    cudaFree(dr);
    cudaFree(dn);
    if (e != cudaSuccess) return cuda_fail(e, "philox");
    return PMF_OK;
}

pmf_status pmf_chain_schedule(int N, int NW, int precision, int *out, size_t capacity, size_t *n_written,
                              int *padded)
{
    return pmf_chain_schedule_variant(N, NW, precision, 0, out, capacity, n_written, padded);
}

int pmf_chain_schedule_variants(void) { return kSchedVariants; }

pmf_status pmf_chain_schedule_variant(int N, int NW, int precision, int variant, int *out, size_t capacity,
                                      size_t *n_written, int *padded)
{
    if (N < 4 || N > 1024 || (NW != 4 && NW != 5 && NW != 6 && NW != 8) || (precision != PMF_FP32 && precision != PMF_FP64))
        return fail(PMF_EINVAL, "pmf_chain_schedule: N in [4,1024], NW 4, 5, 6 or 8, precision FP32 or FP64");
    if (variant < 0 || variant >= kSchedVariants) return fail(PMF_EINVAL, "pmf_chain_schedule: bad variant");
    const auto sched = chain_schedule(N, NW, precision == PMF_FP32, variant);
    size_t n = 0;
    for (const auto &v : sched) n += v.size();
    if (n_written) *n_written = n;
    if (padded) *padded = chain_geometry(N).Np;
    if (!out || capacity < 7 * n) return fail(PMF_EINVAL, "pmf_chain_schedule: capacity too small");
    size_t q = 0;
    for (int w = 0; w < NW; ++w)
        for (const UnitDesc &u : sched[w]) {
            int *o = out + 7 * q++;
            o[0] = w; o[1] = u.I1; o[2] = u.I2; o[3] = u.J; o[4] = u.kind; o[5] = u.near1; o[6] = u.near2;
        }
    return PMF_OK;
}

pmf_status pmf_chain_forces(pmf_system *sys, int chain, const double *pos, double lambda, double k, double *forces)
{
    if (!sys || !pos || !forces) return fail(PMF_EINVAL, "null argument");
    if (sys->model != PMF_MODEL_CHAIN || chain < 0 || chain >= (int)sys->chains.size())
        return fail(PMF_EINVAL, "not a chain system / bad chain index");
    ChainModel &m = *sys->chains[chain];
    const int N = m.n_beads(), Np = m.n_padded();
    const bool dbl = m.precision() == PMF_FP64;
    // a one-replica state holding pos, zero velocity, run for zero steps
    const size_t es = dbl ? sizeof(double) : sizeof(float);
    std::vector<unsigned char> st(m.state_bytes_per_replica(), 0);
    for (int b = 0; b < Np; ++b)
        for (int a = 0; a < 3; ++a) {
            const double v = b < N ? pos[3 * b + a] : (a == 0 ? 1.0e4 + 100.0 * b : 1.0e4);
            if (dbl) reinterpret_cast<double *>(st.data())[(size_t)b * 4 + a] = v;
            else reinterpret_cast<float *>(st.data())[(size_t)b * 4 + a] = (float)v;
        }
    (void)es;
    struct Tmp {
        void *state = nullptr;
        double *lam = nullptr, *f = nullptr;
        long long *ns = nullptr;
        int *err = nullptr;
        float *x = nullptr;
        ~Tmp() { cudaFree(state); cudaFree(lam); cudaFree(f); cudaFree(ns); cudaFree(err); cudaFree(x); }
    } t;
    long long one[4] = {1, 0, 0, 1};
    CK(upload(reinterpret_cast<unsigned char **>(&t.state), st.data(), st.size()), "upload state");
    CK(upload(&t.lam, &lambda, 1), "upload lambda");
    CK(upload(&t.ns, one, 4), "upload counts");
    CK(cudaMalloc(&t.f, sizeof(double) * 3 * N), "alloc forces");
    CK(cudaMalloc(&t.x, sizeof(float)), "alloc");
    CK(cudaMalloc(&t.err, sizeof(int)), "alloc");
    CK(cudaMemset(t.err, 0, sizeof(int)), "clear");
    RunLaunch L;
    L.state = t.state;
    L.xout = t.x;
    L.lambda = t.lam;
    L.nsteps_w = t.ns;
    L.nequil_w = t.ns + 1;
    L.off_w = t.ns + 2;
    L.tw = t.ns + 3;
    L.err = t.err;
    L.force_out = t.f;
    L.step_begin = 1;  // resume from the given state: no velocity draw
    L.step_end = 1;
    L.replicas = 1;
    L.stride = 1;
    L.n_blocks = 1;
    L.k = k;
    L.kT = 1.0;
    L.dt = 1e-3;
    L.gamma = 1.0;
    cudaError_t e = m.launch(L, g_stream);
    if (e != cudaSuccess) return cuda_fail(e, "forces");
    CK(cudaMemcpyAsync(forces, t.f, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, g_stream), "copy forces");
    CK(cudaStreamSynchronize(g_stream), "sync");
    return PMF_OK;
}

}  // extern "C"
