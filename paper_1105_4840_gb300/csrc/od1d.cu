// Overdamped Langevin particle in the 1D double well, FP64, one thread per
// (window, replica): the PPP of Sec. III (ii) on the model
// H(lambda, x) = a (x^2 - 1)^2 + k/2 (x - lambda)^2 (kT units).
//   x_{n+1} = x_n + F(x_n) dt / gamma + sqrt(2 kT dt / gamma) xi_n,
// xi_n = normal (n mod 4) of the Philox block (0, uid, n div 4, 0).
#include "common.cuh"
#include "internal.h"

namespace pmf {

struct Od1dArgs {
    double a, x0, k, kT, dt, gamma;
    const double *lambda;
    const long long *nsteps_w, *nequil_w, *off_w, *tw;
    double *state;
    const double *start;
    float *xout;
    int *err;
    long long step_begin, step_end;
    int replicas, stride, n_rep;
    uint32_t uid_base;
    unsigned long long seed;
    int sequential, n_windows;  // sequential protocol: each thread visits every window
    long long window_steps;     //   for window_steps steps, in order
    double *wout;               // constant-velocity pulling: work at the records
    double smd_vdt;             //   trap advance per step after the equilibration
};

// Sequential pulling protocol (Sec. III (i)): simulation r visits the
// windows in order, window w covering steps [w tau, (w + 1) tau) of one
// continuous run; equilibration and sampling count from the window's start.
__device__ void od1d_sequential(const Od1dArgs &a, int r)
{
    const uint32_t uid = a.uid_base + (uint32_t)r;
    const double amp = sqrt(2.0 * a.kT * a.dt / a.gamma);
    double x = a.start ? a.start[r] : a.x0;
    for (int w = 0; w < a.n_windows; ++w) {
        const double lam = a.lambda[w];
        const long long origin = (long long)w * a.window_steps, nequil = a.nequil_w[w];
        const long long base = a.off_w[w] + (long long)r * a.tw[w];
        Normal4<double> n = philox_normals<double>(a.seed, 0u, uid, (uint32_t)(origin >> 2), kTagOStep);
        for (long long step = origin; step < origin + a.window_steps; ++step) {
            const int lane = (int)(step & 3);
            if (lane == 0) n = philox_normals<double>(a.seed, 0u, uid, (uint32_t)(step >> 2), kTagOStep);
            const double xi = lane == 0 ? n.n0 : (lane == 1 ? n.n1 : (lane == 2 ? n.n2 : n.n3));
            const double f = -4.0 * a.a * x * (x * x - 1.0) - a.k * (x - lam);
            x = x + f * a.dt / a.gamma + amp * xi;
            const long long done = step + 1 - origin;
            if (done > nequil && (done - nequil) % a.stride == 0) a.xout[base + (done - nequil) / a.stride - 1] = (float)x;
        }
    }
    if (!isfinite(x)) atomicOr(a.err, kErrNonFinite);
    a.state[r] = x;
}

__global__ void od1d_kernel(const Od1dArgs a)
{
    const int rep = blockIdx.x * blockDim.x + threadIdx.x;
    if (rep >= a.n_rep) return;
    if (a.sequential) {
        od1d_sequential(a, rep);
        return;
    }
    const int w = rep / a.replicas, r = rep % a.replicas;
    const uint32_t uid = a.uid_base + (uint32_t)rep;
    const double lam = a.lambda[w];
    const long long nsteps = a.nsteps_w[w], nequil = a.nequil_w[w];
    const long long s0 = a.step_begin, s1 = a.step_end < nsteps ? a.step_end : nsteps;
    if (s0 >= s1) return;
    double x = s0 == 0 ? (a.start ? a.start[rep] : a.x0) : a.state[rep];
    const double amp = sqrt(2.0 * a.kT * a.dt / a.gamma);
    const long long base = a.off_w[w] + (long long)r * a.tw[w];
    Normal4<double> n = philox_normals<double>(a.seed, 0u, uid, (uint32_t)(s0 >> 2), kTagOStep);
    // constant-velocity pulling: before step m > nequil the trap moves to
    // lam + vdt (m - nequil) with the work of Eq. (9) at the current x
    // (one launch covers the whole run, so the work lives in a register)
    double lam_now = lam, W = 0.0;
    for (long long step = s0; step < s1; ++step) {
        if (a.wout && step > nequil) {
            const double ln = lam + a.smd_vdt * (double)(step - nequil);
            W += 0.5 * a.k * (ln - lam_now) * (ln + lam_now - 2.0 * x);
            lam_now = ln;
        }
        const int lane = (int)(step & 3);
        if (lane == 0) n = philox_normals<double>(a.seed, 0u, uid, (uint32_t)(step >> 2), kTagOStep);
        const double xi = lane == 0 ? n.n0 : (lane == 1 ? n.n1 : (lane == 2 ? n.n2 : n.n3));
        const double f = -4.0 * a.a * x * (x * x - 1.0) - a.k * (x - lam_now);
        x = x + f * a.dt / a.gamma + amp * xi;
        const long long done = step + 1;
        if (done > nequil && (done - nequil) % a.stride == 0) {
            a.xout[base + (done - nequil) / a.stride - 1] = (float)x;
            if (a.wout) a.wout[base + (done - nequil) / a.stride - 1] = W;
        }
    }
    if (!isfinite(x)) atomicOr(a.err, kErrNonFinite);
    a.state[rep] = x;
}

cudaError_t od1d_launch(const Od1dParams &m, const RunLaunch &L, int n_rep, cudaStream_t st)
{
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
    a.step_begin = L.step_begin;
    a.step_end = L.step_end;
    a.replicas = L.replicas;
    a.stride = L.stride;
    a.n_rep = n_rep;
    a.uid_base = L.uid_base;
    a.seed = L.seed;
    a.sequential = L.sequential ? 1 : 0;
    a.window_steps = L.window_steps;
    a.wout = L.wout;
    a.smd_vdt = L.smd_vdt;
    if (L.wout && L.step_begin != 0) return cudaErrorInvalidValue;  // pulled runs are one launch
    a.n_windows = L.sequential ? (int)(L.step_end / L.window_steps) : 0;
    if (L.sequential && (L.window_steps < 1 || L.step_begin != 0)) return cudaErrorInvalidValue;
    const int threads = 128;
    od1d_kernel<<<(n_rep + threads - 1) / threads, threads, 0, st>>>(a);
    return cudaGetLastError();
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
