// Work distributions from binned reaction-coordinate distributions (App. C).
//
// rho_i: the samples of window i counted into n_x bins of width dx (integer
// atomics, so the counts are exact and the result deterministic).  Omega_i
// lives on work bins W = b dW, b = -M..M; Omega_1 is all at W = 0 and
//   Omega_{i+1}(b') = sum_j rho_i(j) Omega_i(b' - shift_i(j)),
// shift_i(j) = round(w_i(x_j) / dW) with w_i of Eq. (9) at the bin centre
// x_j (or, for the rule as printed, floor(w_i / dW) at the bin's left edge,
// with the W = 0 bin smoothed after every step).  Because shift_i is monotone
// in j, the x bins sharing one shift form a contiguous run: g_i(s), the
// probability of shift s, is summed over that run (found by bisection), and
// Omega_{i+1} = Omega_i * g_i is a direct 1D convolution over the supports.
#include <math.h>

#include "../../include/pmf.h"
#include "common.cuh"
#include "internal.h"

namespace pmf {

namespace {

// Rounded operations (no contraction into FMA) so the bin positions match a
// plain evaluation x_lo + (j + 1/2) dx step by step.
__device__ __forceinline__ long long bin_shift(const HistStep &h, long long j)
{
    const double x = __dadd_rn(h.x_lo, __dmul_rn(__dadd_rn((double)j, h.left_edge ? 0.0 : 0.5), h.dx));
    const double w = h.hk * h.d * (h.lsum - 2.0 * x);
    return (long long)floor(h.left_edge ? w / h.dw : w / h.dw + 0.5);
}

__global__ void count_kernel(const float *x, const long long *off_w, const long long *tw, int replicas, double x_lo,
                             double dx, int n_x, unsigned long long *cnt, unsigned long long *outside, int *jmin,
                             int *jmax)
{
    const int w = blockIdx.y;
    const long long n = tw[w] * replicas;
    const float *xs = x + off_w[w];
    unsigned long long *c = cnt + (size_t)w * n_x;
    int lo = 0x7fffffff, hi = -1;
    unsigned long long out = 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const double j = floor(((double)xs[t] - x_lo) / dx);
        if (j >= 0.0 && j < (double)n_x) {
            const int ji = (int)j;
            atomicAdd(c + ji, 1ull);
            lo = ji < lo ? ji : lo;
            hi = ji > hi ? ji : hi;
        } else {
            ++out;
        }
    }
    if (out) atomicAdd(outside + w, out);
    if (hi >= 0) {
        atomicMin(jmin + w, lo);
        atomicMax(jmax + w, hi);
    }
}

// g[s - gmin] for s in [gmin, gmax]: probability of work shift s
__global__ void shift_prob_kernel(const HistStep h, const unsigned long long *cnt, double inv_n, double *g)
{
    const long long s = h.gmin + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s > h.gmax) return;
    // key(j) non-decreasing in j: -shift when the work falls with x (d > 0)
    const bool dec = h.d > 0.0;
    auto key = [&](long long j) { return dec ? -bin_shift(h, j) : bin_shift(h, j); };
    const long long target = dec ? -s : s;
    long long a = h.jmin, b = h.jmax + 1;  // first j with key >= target
    while (a < b) {
        const long long m = (a + b) >> 1;
        if (key(m) < target) a = m + 1;
        else b = m;
    }
    unsigned long long sum = 0;
    for (long long j = a; j <= h.jmax && key(j) == target; ++j) sum += cnt[j];
    g[s - h.gmin] = (double)sum * inv_n;
}

// out[b] = sum_s g[s] in[b - s] over the supports; b indexes -M..M at b + M
__global__ void conv_kernel(const double *in, long long in_lo, long long in_hi, const double *g, long long gmin,
                            long long gmax, double *out, long long out_lo, long long out_hi, long long M)
{
    const long long b = out_lo + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b > out_hi) return;
    long long s0 = b - in_hi > gmin ? b - in_hi : gmin;
    long long s1 = b - in_lo < gmax ? b - in_lo : gmax;
    double acc = 0.0;
    for (long long s = s0; s <= s1; ++s) acc += g[s - gmin] * in[b - s + M];
    out[b + M] = acc;
}

__global__ void smooth_zero_kernel(double *om, long long M)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) om[M] = 0.5 * (om[M - 1] + om[M + 1]);
}

constexpr int kStatThreads = 256;

template <typename F> __device__ double block_reduce(double v, double *red, F op, double ident)
{
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < kStatThreads / 32 ? red[l] : ident;
        for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (l == 0) red[0] = v;
    }
    __syncthreads();
    return red[0];
}

// per window: total, min W over non-zero bins, JE, mean, variance, Q
__global__ void __launch_bounds__(kStatThreads) omega_stats_kernel(const double *om, long long M, double dw, double kT,
                                                                   const long long *sup, double *stats)
{
    __shared__ double red[kStatThreads / 32];
    const int i = blockIdx.x;
    const double *p = om + (size_t)i * (2 * M + 1);
    const long long lo = sup[2 * i], hi = sup[2 * i + 1];
    const auto add = [](double a, double b) { return a + b; };
    const auto mn = [](double a, double b) { return fmin(a, b); };
    double tot = 0, wmin = INFINITY, q = 0;
    for (long long b = lo + threadIdx.x; b <= hi; b += kStatThreads) {
        const double v = p[b + M];
        tot += v;
        if (v > 0.0) {
            wmin = fmin(wmin, (double)b * dw);
            q += 1.0;
        }
    }
    tot = block_reduce(tot, red, add, 0.0);
    wmin = block_reduce(wmin, red, mn, INFINITY);
    q = block_reduce(q, red, add, 0.0);
    double se = 0, sw = 0;
    for (long long b = lo + threadIdx.x; b <= hi; b += kStatThreads) {
        const double v = p[b + M], W = (double)b * dw;
        if (v > 0.0) se += v * exp(-(W - wmin) / kT);
        sw += v * W;
    }
    se = block_reduce(se, red, add, 0.0);
    const double mean = block_reduce(sw, red, add, 0.0) / tot;
    double sv = 0;
    for (long long b = lo + threadIdx.x; b <= hi; b += kStatThreads) {
        const double d = (double)b * dw - mean;
        sv += p[b + M] * d * d;
    }
    const double var = block_reduce(sv, red, add, 0.0) / tot;
    if (threadIdx.x == 0) {
        stats[4 * i + 0] = wmin - kT * log(se / tot);
        stats[4 * i + 1] = q > 1.0 ? var / q + var * var / (2.0 * kT * kT * (q - 1.0)) : 0.0;
        stats[4 * i + 2] = tot;
        stats[4 * i + 3] = q;
    }
}

}  // namespace

cudaError_t hist_count_launch(const float *x, const long long *off_w, const long long *tw, int n_windows, int replicas,
                              double x_lo, double dx, int n_x, unsigned long long *cnt, unsigned long long *outside,
                              int *jmin, int *jmax, cudaStream_t st)
{
    count_kernel<<<dim3(64, n_windows), 256, 0, st>>>(x, off_w, tw, replicas, x_lo, dx, n_x, cnt, outside, jmin, jmax);
    return cudaGetLastError();
}

// Host copy of the shift of bin j (used only to bound the supports; they
// are widened by one on each side, so a last-bit difference cannot matter).
long long hist_shift_host(const HistStep &h, long long j)
{
    const double x = h.x_lo + ((double)j + (h.left_edge ? 0.0 : 0.5)) * h.dx;
    const double w = h.hk * h.d * (h.lsum - 2.0 * x);
    return (long long)floor(h.left_edge ? w / h.dw : w / h.dw + 0.5);
}

cudaError_t hist_step_launch(const HistStep &h, const unsigned long long *cnt_w, double inv_n, double *g,
                             const double *in, long long in_lo, long long in_hi, double *out, long long out_lo,
                             long long out_hi, long long M, cudaStream_t st)
{
    const long long ng = h.gmax - h.gmin + 1;
    shift_prob_kernel<<<(unsigned)((ng + 127) / 128), 128, 0, st>>>(h, cnt_w, inv_n, g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (out_hi >= out_lo) {
        const long long nb = out_hi - out_lo + 1;
        conv_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(in, in_lo, in_hi, g, h.gmin, h.gmax, out, out_lo,
                                                                  out_hi, M);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (h.left_edge) {
        smooth_zero_kernel<<<1, 32, 0, st>>>(out, M);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t hist_stats_launch(const double *om, int n_windows, long long M, double dw, double kT, const long long *sup,
                              double *stats, cudaStream_t st)
{
    omega_stats_kernel<<<n_windows, kStatThreads, 0, st>>>(om, M, dw, kT, sup, stats);
    return cudaGetLastError();
}

}  // namespace pmf
