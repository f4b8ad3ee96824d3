// Learned window placement, device side: overlap of adjacent predicted x
// distributions and seeding of inserted windows.
//
// The paper's criterion (Sec. III after Eq. (9), Sec. IV B, Sec. V (iii)):
// adjacent x distributions must overlap comparably to their spread.  With
// the surrogate's Gaussian prediction N(mu_i, sigma_i^2) per window the
// overlap coefficient OVL = int min(p_i, p_{i+1}) has a closed form: the two
// pdfs cross where their log-densities agree (a quadratic in x), and between
// the crossings the wider Gaussian is the smaller pdf.
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace pmf {

__device__ __forceinline__ double phi_cdf(double z) { return 0.5 * erfc(-z * 0.70710678118654752440); }

__device__ double gaussian_ovl(double m1, double s1, double m2, double s2)
{
    if (fabs(s1 - s2) < 1e-12 * fmax(s1, s2)) return 2.0 * phi_cdf(-fabs(m1 - m2) / (2.0 * s1));
    const double a = 1.0 / (2 * s2 * s2) - 1.0 / (2 * s1 * s1);
    const double b = m1 / (s1 * s1) - m2 / (s2 * s2);
    const double c = m2 * m2 / (2 * s2 * s2) - m1 * m1 / (2 * s1 * s1) + log(s2 / s1);
    const double disc = fmax(b * b - 4 * a * c, 0.0);
    double r1 = (-b - sqrt(disc)) / (2 * a), r2 = (-b + sqrt(disc)) / (2 * a);
    if (r1 > r2) { const double t = r1; r1 = r2; r2 = t; }
    const double mw = s1 > s2 ? m1 : m2, sw = s1 > s2 ? s1 : s2;
    const double mn = s1 > s2 ? m2 : m1, sn = s1 > s2 ? s2 : s1;
    const double inside = phi_cdf((r2 - mw) / sw) - phi_cdf((r1 - mw) / sw);
    const double outside = phi_cdf((r1 - mn) / sn) + (1.0 - phi_cdf((r2 - mn) / sn));
    return inside + outside;
}

__global__ void overlap_kernel(const double *mu, const double *log_var, int n, double *ovl)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i + 1 >= n) return;
    ovl[i] = gaussian_ovl(mu[i], exp(0.5 * log_var[i]), mu[i + 1], exp(0.5 * log_var[i + 1]));
}

cudaError_t overlap_launch(const double *mu, const double *log_var, int n, double *ovl, cudaStream_t st)
{
    if (n < 2) return cudaSuccess;
    overlap_kernel<<<(n + 127) / 128, 128, 0, st>>>(mu, log_var, n, ovl);
    return cudaGetLastError();
}

// Measured Gaussian moments of the windows (the gate that decides whether a
// round needs the surrogate at all): block w reads the replicas x T_w
// samples of window w of a merged store and writes mu[w] = their mean and
// log_var[w] = log of their population variance, both in FP64 (two passes:
// the mean, then the mean squared deviation from it).
constexpr int kMomentThreads = 256;

__device__ double moment_block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();  // red may still be read by a previous call
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0;
    for (int i = 0; i < kMomentThreads / 32; ++i) t += red[i];
    return t;
}

__global__ void __launch_bounds__(kMomentThreads) moments_kernel(const float *x, const long long *off,
                                                                 const long long *tw, int replicas, double *mu,
                                                                 double *log_var)
{
    __shared__ double red[kMomentThreads / 32];
    const int w = blockIdx.x;
    const long long n = tw[w] * replicas;
    const float *xw = x + off[w];
    double s = 0;
    for (long long i = threadIdx.x; i < n; i += kMomentThreads) s += (double)xw[i];
    const double m = n > 0 ? moment_block_sum(s, red) / (double)n : NAN;
    double q = 0;
    for (long long i = threadIdx.x; i < n; i += kMomentThreads) {
        const double d = (double)xw[i] - m;
        q += d * d;
    }
    const double v = n > 0 ? moment_block_sum(q, red) / (double)n : NAN;
    if (threadIdx.x == 0) {
        mu[w] = m;
        log_var[w] = log(v);
    }
}

cudaError_t moments_launch(const float *x, const long long *off, const long long *tw, int replicas, int n,
                           double *mu, double *log_var, cudaStream_t st)
{
    if (n < 1) return cudaSuccess;
    moments_kernel<<<n, kMomentThreads, 0, st>>>(x, off, tw, replicas, mu, log_var);
    return cudaGetLastError();
}

// Seeding: block q fills the start states of inserted window q.  Its M
// candidates are stored end states (positions of M replicas of the two
// neighbouring windows); replica r starts from the candidate of rank r mod M
// when candidates are ordered by |x_final - target_q| (ties by index).  A
// NaN target keeps the candidates in their order (a window continued from
// its own replicas' end states).
template <typename R>
__global__ void seed_kernel(const SeedJob *jobs, int N, int Np, int replicas, int max_cand, double *start,
                            int *choice, double *cand_x)
{
    extern __shared__ double dist[];  // [M]
    const SeedJob &J = jobs[blockIdx.x];
    const int M = J.n_cand;
    for (int c = threadIdx.x; c < M; c += blockDim.x) {
        double x;
        if (N > 0) {
            const R *p = reinterpret_cast<const R *>(J.cand[c]);  // positions, 4 values per bead
            const double dx = (double)p[4 * (N - 1) + 0] - (double)p[0];
            const double dy = (double)p[4 * (N - 1) + 1] - (double)p[1];
            const double dz = (double)p[4 * (N - 1) + 2] - (double)p[2];
            x = sqrt(dx * dx + dy * dy + dz * dz);
        } else {
            x = *reinterpret_cast<const double *>(J.cand[c]);
        }
        dist[c] = fabs(x - J.target);
        if (cand_x) cand_x[(size_t)blockIdx.x * max_cand + c] = x;
    }
    __syncthreads();
    const bool keep_order = !(J.target == J.target);  // NaN target: candidate c to replica c (continuation)
    for (int c = threadIdx.x; c < M; c += blockDim.x) {
        int rank = 0;
        if (keep_order) rank = c;
        else
            for (int d = 0; d < M; ++d) rank += (dist[d] < dist[c]) || (dist[d] == dist[c] && d < c);
        for (int r = rank; r < replicas; r += M) {
            if (choice) choice[(size_t)blockIdx.x * replicas + r] = c;
            double *out = start + ((size_t)blockIdx.x * replicas + r) * (N > 0 ? 3 * (size_t)N : 1);
            if (N > 0) {
                const R *p = reinterpret_cast<const R *>(J.cand[c]);
                for (int b = 0; b < N; ++b)
                    for (int k = 0; k < 3; ++k) out[3 * b + k] = (double)p[4 * b + k];
            } else {
                out[0] = *reinterpret_cast<const double *>(J.cand[c]);
            }
        }
    }
}

cudaError_t seed_launch(const SeedJob *jobs, int n_jobs, int max_cand, int N, int Np, int replicas, bool fp64,
                        double *start, int *choice, double *cand_x, cudaStream_t st)
{
    if (n_jobs == 0) return cudaSuccess;
    const size_t smem = sizeof(double) * (size_t)max_cand;
    if (fp64 || N == 0)
        seed_kernel<double><<<n_jobs, 128, smem, st>>>(jobs, N, Np, replicas, max_cand, start, choice, cand_x);
    else
        seed_kernel<float><<<n_jobs, 128, smem, st>>>(jobs, N, Np, replicas, max_cand, start, choice, cand_x);
    return cudaGetLastError();
}

}  // namespace pmf
