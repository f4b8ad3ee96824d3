// Overdamped Langevin particle in the 1D double well, FP64, one thread per
// simulation: the PPP of Sec. III (ii) (and the sequential protocol and
// constant-velocity pulling) on the model
// H(lambda, x) = a (x^2 - 1)^2 + k/2 (x - lambda)^2 (kT units).
//   x_{n+1} = x_n + F(x_n) dt / gamma + sqrt(2 kT dt / gamma) xi_n,
// F = -dH/dx, xi_n = normal (n mod 4) of the Philox block (0, uid, n div 4, 0).
// Regrouped, x_{n+1} = x_n (cA x_n^2 + cB) + q_n with cA = -4a dt/gamma,
// cB = 1 + (4a - k) dt/gamma and q_n = k lambda_n dt/gamma + amp xi_n.  q_n
// does not depend on the trajectory, so a parallel pre-pass computes it for
// a block of steps of every simulation; the sequential integration then costs
// three FP64 operations per step, the rate at which this GPU's FP64 unit
// retires them bounding a few hundred simulations.
#include "common.cuh"
#include "internal.h"

namespace pmf {

struct Od1dArgs {
    double a, x0, k, kT, dt, gamma;
    const double *lambda;
    const long long *nsteps_w, *nequil_w, *off_w, *tw;
    double *state;              // [n_rep][2]: x and the accumulated pulling work
    const double *start;
    float *xout;
    int *err;
    long long c0, c1;           // this launch's steps
    int replicas, stride, n_rep;
    uint32_t uid_base;
    unsigned long long seed;
    int sequential;             // sequential protocol: window = step / window_steps
    long long window_steps;
    double *wout;               // constant-velocity pulling: work at the records
    double smd_vdt;             //   trap advance per step after the equilibration
    const double *noise;        // [c1 - c0][n_rep] q_n of this launch's steps
};

// Trap centre during step n of simulation rep: its window's lambda (the
// window of step n in the sequential protocol), or, when pulled, lambda_1
// advanced by vdt per step after the equilibration.
__device__ __forceinline__ double trap_centre(const Od1dArgs &a, int rep, long long n)
{
    if (a.wout) {
        const long long nequil = a.nequil_w[0];
        return n > nequil ? a.lambda[0] + a.smd_vdt * (double)(n - nequil) : a.lambda[0];
    }
    return a.lambda[a.sequential ? (int)(n / a.window_steps) : rep / a.replicas];
}

// q_n of every simulation for steps [c0, c1), one Philox block (four steps
// of one simulation) per thread, stored [n - c0][rep].
__global__ void od1d_noise_kernel(const Od1dArgs a, double *q)
{
    const long long nb = (a.c1 - a.c0 + 3) >> 2;  // c0 is a multiple of 4
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nb * a.n_rep) return;
    const int rep = (int)(i % a.n_rep);
    const long long blk = i / a.n_rep;
    const long long n0 = a.c0 + 4 * blk;
    const Normal4<double> z =
        philox_normals<double>(a.seed, 0u, a.uid_base + (uint32_t)rep, (uint32_t)(n0 >> 2), kTagOStep);
    const double v[4] = {z.n0, z.n1, z.n2, z.n3};
    const double dtg = a.dt / a.gamma, amp = sqrt(2.0 * a.kT * dtg), ck = a.k * dtg;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const long long n = n0 + l;
        if (n < a.c1) q[(n - a.c0) * a.n_rep + rep] = fma(amp, v[l], ck * trap_centre(a, rep, n));
    }
}

// One thread per simulation, steps [c0, c1): the parallel protocol (window
// rep / R throughout), the sequential protocol (window = step / tau, Sec.
// III (i)) or constant-velocity pulling (the trap at lambda_1 + vdt (n -
// n_equil) from step n_equil on, the move before step n doing the work of
// Eq. (9) at the current x).
// First `done` count (steps completed in the window) > from at which a sample
// is recorded: nequil + m stride, m >= 1.
__device__ __forceinline__ long long next_sample(long long from, long long nequil, int stride)
{
    const long long m = from < nequil + stride ? 1 : (from - nequil) / stride + 1;
    return nequil + m * stride;
}

__global__ void od1d_kernel(const Od1dArgs a)
{
    const int rep = blockIdx.x * blockDim.x + threadIdx.x;
    if (rep >= a.n_rep) return;
    const int r = a.sequential ? rep : rep % a.replicas;
    int w = a.sequential ? (int)(a.c0 / a.window_steps) : rep / a.replicas;
    long long c1 = a.c1;
    if (!a.sequential) c1 = c1 < a.nsteps_w[w] ? c1 : a.nsteps_w[w];
    if (a.c0 >= c1) return;
    double x = a.c0 == 0 ? (a.start ? a.start[rep] : a.x0) : a.state[2 * rep];
    double W = a.c0 == 0 ? 0.0 : a.state[2 * rep + 1];
    const double lam1 = a.lambda[0], dtg = a.dt / a.gamma;
    const double cA = -4.0 * a.a * dtg, cB = 1.0 + (4.0 * a.a - a.k) * dtg;
    // per-window quantities, refreshed when a sequential run enters a window
    long long origin = a.sequential ? (long long)w * a.window_steps : 0;
    long long win_end = a.sequential ? origin + a.window_steps : c1;
    long long nequil = a.nequil_w[w];
    double lam = a.lambda[w];
    long long base = a.off_w[w] + (long long)r * a.tw[w];
    long long next = next_sample(a.c0 - origin, nequil, a.stride);  // in the window's step count
    if (a.wout && a.c0 - 1 > nequil) lam = lam1 + a.smd_vdt * (double)(a.c0 - 1 - nequil);  // pulled so far
    // q_n in blocks of kPre steps, the next block's loads issued before the
    // current block is integrated (the dependent steps are short; an L2 load
    // per step would otherwise stall every step)
    constexpr int kPre = 8;
    const double *xi = a.noise + rep;
    double cur[kPre], nxt[kPre];
#pragma unroll
    for (int j = 0; j < kPre; ++j) cur[j] = a.c0 + j < c1 ? xi[(long long)j * a.n_rep] : 0.0;
    for (long long n0 = a.c0; n0 < c1; n0 += kPre) {
#pragma unroll
        for (int j = 0; j < kPre; ++j) {
            const long long m = n0 + kPre + j;
            nxt[j] = m < c1 ? xi[(m - a.c0) * a.n_rep] : 0.0;
        }
#pragma unroll
        for (int j = 0; j < kPre; ++j) {
        const long long n = n0 + j;
        if (n >= c1) break;
        if (n == win_end) {  // sequential protocol: the trap moves to the next window
            ++w;
            origin = n;
            win_end = n + a.window_steps;
            nequil = a.nequil_w[w];
            lam = a.lambda[w];
            base = a.off_w[w] + (long long)r * a.tw[w];
            next = next_sample(0, nequil, a.stride);
        }
        if (a.wout && n > nequil) {
            const double lo = lam;
            lam = lam1 + a.smd_vdt * (double)(n - nequil);
            W += 0.5 * a.k * (lam - lo) * (lam + lo - 2.0 * x);
        }
        x = fma(x, fma(cA, x * x, cB), cur[j]);
        if (n + 1 - origin == next) {
            const long long at = base + (next - nequil) / a.stride - 1;
            a.xout[at] = (float)x;
            if (a.wout) a.wout[at] = W;
            next += a.stride;
        }
        }
#pragma unroll
        for (int j = 0; j < kPre; ++j) cur[j] = nxt[j];
    }
    if (!isfinite(x)) atomicOr(a.err, kErrNonFinite);
    a.state[2 * rep] = x;
    a.state[2 * rep + 1] = W;
}

long long od1d_noise_steps(int n_rep)
{
    // at most 2^23 normals (64 MB) per launch, between 64 and 8192 steps
    long long c = (1LL << 23) / (n_rep > 0 ? n_rep : 1);
    c = c < 64 ? 64 : (c > 8192 ? 8192 : c);
    return c & ~3LL;
}

cudaError_t od1d_launch(const Od1dParams &m, const RunLaunch &L, int n_rep, cudaStream_t st)
{
    if (L.noise == nullptr || L.noise_steps < 4 || (L.noise_steps & 3) != 0 || (L.step_begin & 3) != 0)
        return cudaErrorInvalidValue;
    if (L.sequential && L.window_steps < 1) return cudaErrorInvalidValue;
    Od1dArgs a{};
    a.a = m.a;
    a.x0 = m.x0;
    a.k = L.k;
    a.kT = L.kT;
    a.dt = L.dt;
    a.gamma = L.gamma;
    a.lambda = L.lambda;
    a.nsteps_w = L.nsteps_w;
    a.nequil_w = L.nequil_w;
    a.off_w = L.off_w;
    a.tw = L.tw;
    a.state = reinterpret_cast<double *>(L.state);
    a.start = L.start;
    a.xout = L.xout;
    a.err = L.err;
    a.replicas = L.replicas;
    a.stride = L.stride;
    a.n_rep = n_rep;
    a.uid_base = L.uid_base;
    a.seed = L.seed;
    a.sequential = L.sequential ? 1 : 0;
    a.window_steps = L.window_steps;
    a.wout = L.wout;
    a.smd_vdt = L.smd_vdt;
    a.noise = L.noise;
    // few simulations: spread them over the SMs (one warp each) rather than
    // packing them into a few CTAs; many: 128 threads per CTA
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cudaGetLastError();
    const int per_sm = (n_rep + sms - 1) / sms;
    const int threads = per_sm <= 32 ? 32 : (per_sm <= 64 ? 64 : 128);
    for (long long c0 = L.step_begin; c0 < L.step_end; c0 += L.noise_steps) {
        const long long c1 = c0 + L.noise_steps < L.step_end ? c0 + L.noise_steps : L.step_end;
        const long long cells = ((c1 - c0 + 3) >> 2) * n_rep;
        a.c0 = c0;
        a.c1 = c1;
        od1d_noise_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(a, L.noise);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        od1d_kernel<<<(n_rep + threads - 1) / threads, threads, 0, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Philox test hook: the same generator and FP32 Box-Muller as the integrator.
__global__ void philox_kernel(unsigned long long seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int n,
                              uint32_t *raw, float *normals)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Ctr4 b = philox4x32_10(Ctr4{c0 + (uint32_t)i, c1, c2, c3}, (uint32_t)seed, (uint32_t)(seed >> 32));
    if (raw) {
        raw[4 * i + 0] = b.a;
        raw[4 * i + 1] = b.b;
        raw[4 * i + 2] = b.c;
        raw[4 * i + 3] = b.d;
    }
    if (normals) {
        const Normal4<float> z = box_muller(b, 0.0f);
        normals[4 * i + 0] = z.n0;
        normals[4 * i + 1] = z.n1;
        normals[4 * i + 2] = z.n2;
        normals[4 * i + 3] = z.n3;
    }
}

cudaError_t philox_launch(unsigned long long seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int n,
                          uint32_t *raw, float *normals, cudaStream_t st)
{
    philox_kernel<<<(n + 255) / 256, 256, 0, st>>>(seed, c0, c1, c2, c3, n, raw, normals);
    return cudaGetLastError();
}

}  // namespace pmf
