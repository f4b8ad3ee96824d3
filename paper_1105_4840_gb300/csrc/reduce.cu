// FP64 reductions of the recorded x samples into the paper's estimators.
//
// Stage 1 (one CTA per (window i, replica r), two passes over the samples):
//   work increments of Eq. (9),
//   w = k/2 (lambda_{i+1} - lambda_i)(lambda_{i+1} + lambda_i - 2 x),
//   the replica's minimum m_ir, the max-shifted exponential sum
//   S_ir = sum exp(-(w - m_ir)/kT) (Eq. (12)), and the shifted moments
//   sum (x - lambda_i), sum (x - lambda_i)^2.
// Stage 2 (one CTA per window): merge the replicas (log-sum-exp aware),
//   the per-window JE increment, the Eq. (14) and Eq. (13) increments and
//   the delete-one-replica jackknife.
// Stage 3 (one thread): prefix sums over windows into the profiles and the
//   combined estimate of Sec. V.
// The windows are independent (Sec. II: rho(W_mech) is the product of the
// rho(x_i)), so the average of exp(-W_mech/kT) over all combinations of
// samples is the product of the per-window averages.
#include <math.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace pmf {

struct Partial {
    double m, S, n, sdx, sdx2;
};
static_assert(sizeof(Partial) == kPartialDoubles * sizeof(double), "partials are exported as 5 doubles");
struct WindowOut {
    double je, fl, g, wmean, varw, n, jk_je, jk_fl, mean, var;
};

__device__ __forceinline__ void neumaier(double &s, double &c, double v)
{
    const double t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
}

template <int NT> __device__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int q = 0; q < NT / 32; ++q) t += red[q];
        red[NT / 32] = t;
    }
    __syncthreads();
    return red[NT / 32];
}

template <int NT> __device__ double block_min(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = red[0];
        for (int q = 1; q < NT / 32; ++q) t = fmin(t, red[q]);
        red[NT / 32] = t;
    }
    __syncthreads();
    return red[NT / 32];
}

constexpr int kPartialThreads = 256;

// ---- the exponential of stage 1 in double-float arithmetic on the FP32 pipe
//
// GB300's FP64 unit retires 1/64 of the FP32 rate, and an FP64 exp per
// sample made stage 1 FP64-bound.  The exponent is linear in x: with the
// work increment w = k/2 (lambda_{i+1} - lambda_i)(lambda_{i+1} + lambda_i - 2x)
// and its minimum at the sample x_ref (the largest x when lambda_{i+1} >
// lambda_i, the smallest otherwise), -(w - min w)/kT = c (x - x_ref) <= 0 with
// c = k (lambda_{i+1} - lambda_i)/kT.  x - x_ref is exact as a pair of floats
// (TwoSum), c (x - x_ref) is formed as a pair of floats, and exp of that pair
// follows Tang's table-driven method (P. T. P. Tang, ACM TOMS 15 (1989)
// 144-157): a = n ln2/32 + r with |r| <= ln2/64, exp(a) = 2^(n div 32)
// 2^((n mod 32)/32) (1 + p(r)), p the Taylor series of e^r - 1 to r^6 (the
// next term is below 2e-18), 2^(j/32) as a pair of floats from the FP64 exp2,
// ln2/32 split in three floats whose first has 12 significant bits so that
// n times it is exact.  The relative error of a term, weighted by its size,
// stays near 1e-14; terms below e^-80 of the largest are dropped (the largest
// is 1).

__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fast_two_sum_f(float a, float b, float &s, float &e)  // |a| >= |b|
{
    s = a + b;
    e = b - (s - a);
}

struct ExpConsts {
    float inv_l;          // 32 / ln 2
    float l1, l2, l3;     // ln2/32 = l1 + l2 + l3, l1 with 12 significant bits
};

__device__ __forceinline__ ExpConsts exp_consts()
{
    // ln 2 as the double nearest to it plus the remainder
    const double ln2_hi = 0.6931471805599453, ln2_lo = 2.319046813846299558e-17;
    const double l = ln2_hi / 32.0;  // exact: a power-of-two scaling
    ExpConsts k;
    k.inv_l = (float)(32.0 / ln2_hi);
    k.l1 = __int_as_float(__float_as_int((float)l) & ~0xFFF);
    const double r1 = l - (double)k.l1;
    k.l2 = (float)r1;
    k.l3 = (float)((r1 - (double)k.l2) + ln2_lo / 32.0);
    return k;
}

// exp(ah + al) for ah + al <= 0 as a pair of floats eh + el (tab: 2^(j/32)
// = tab_hi[j] + tab_lo[j]).
__device__ __forceinline__ void exp_ff(float ah, float al, const ExpConsts &k, const float *tab_hi,
                                       const float *tab_lo, float &eh, float &el)
{
    if (ah < -80.f) {
        eh = el = 0.f;
        return;
    }
    const float kf = rintf(ah * k.inv_l);
    const int n = (int)kf;
    // r = a - n ln2/32: n l1 is exact and close to ah, n l2 exact as p2 + e2
    const float t1 = fmaf(-kf, k.l1, ah);
    const float p2 = kf * k.l2;
    const float e2 = fmaf(kf, k.l2, -p2);
    float rh, rl;
    two_sum_f(t1, -p2, rh, rl);
    rl += (al - e2) - kf * k.l3;
    fast_two_sum_f(rh, rl, rh, rl);
    // e^r - 1 = r + r^2/2 + r^3 (1/6 + r (1/24 + r (1/120 + r/720)))
    const float sh = rh * rh;
    const float sl = fmaf(rh, rh, -sh) + 2.f * rh * rl;
    const float q = rh * sh * fmaf(rh, fmaf(rh, fmaf(rh, 1.f / 720.f, 1.f / 120.f), 1.f / 24.f), 1.f / 6.f);
    float ph, pl;
    two_sum_f(rh, 0.5f * sh, ph, pl);
    pl += (rl + 0.5f * sl) + q;
    fast_two_sum_f(ph, pl, ph, pl);
    // 2^(j/32) (1 + p), then the power of two 2^(n div 32) (exact)
    const int j = n & 31, m = n >> 5;
    const float th = tab_hi[j], tl = tab_lo[j];
    const float uh = th * ph;
    const float ul = fmaf(th, ph, -uh) + (th * pl + tl * ph);
    float hh, hl;
    two_sum_f(th, uh, hh, hl);
    hl += tl + ul;
    const float sc = __int_as_float((m + 127) << 23);
    eh = hh * sc;
    el = hl * sc;
}

// (h, l) += (bh, bl) in double-float arithmetic.
__device__ __forceinline__ void ff_add(float &h, float &l, float bh, float bl)
{
    float s, e;
    two_sum_f(h, bh, s, e);
    e += l + bl;
    fast_two_sum_f(s, e, h, l);
}

// Per-thread sums kept as pairs of floats and flushed into FP64 every
// kFlushSamples terms: within a flush the pair's error stays near
// kFlushSamples x 2^-47 of the partial sum, and the FP64 unit does a few
// operations per flush instead of several per sample.
constexpr int kFlushSamples = 16;

template <int NT> __device__ float block_max_f(float v, float *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float t = red[0];
    for (int q = 1; q < NT / 32; ++q) t = fmaxf(t, red[q]);
    return t;
}

// Per-window constants of stage 1, set once per CTA by one thread (the FP64
// unit is the scarce one: per-thread setup in FP64 would cost more than the
// samples themselves at a few samples per thread).
struct WindowConsts {
    double hkd, ssum;       // w = hkd (ssum - 2 x)
    float ch, cl;           // c = 2 hkd / kT as a pair of floats
    float li_h, li_m, li_l; // lambda_i as three floats
    float sgn;              // +1: x_ref is the largest x, -1: the smallest
    ExpConsts k;
};

__global__ void __launch_bounds__(kPartialThreads) partial_kernel(const ReduceLayout L, Partial *out)
{
    // Two passes over the replica's samples (the second mostly from cache):
    // the extreme x that minimises w, then per thread the exponential sum
    // (terms by exp_ff) and the sums of (x - lambda_i) and its square as
    // pairs of floats flushed into FP64, then trees over the threads.
    __shared__ double red[kPartialThreads / 32 + 1];
    __shared__ float redf[kPartialThreads / 32];
    __shared__ float tab_hi[32], tab_lo[32];
    __shared__ WindowConsts wc;
    const int w = blockIdx.x, r = blockIdx.y;
    const long long T = L.tw[w];
    const float *x = L.x + L.off_w[w] + (long long)r * T;
    if (threadIdx.x < 32) {
        const double t = exp2((double)threadIdx.x / 32.0);
        tab_hi[threadIdx.x] = (float)t;
        tab_lo[threadIdx.x] = (float)(t - (double)(float)t);
    } else if (threadIdx.x == 32) {
        const double li = L.lambda[w];
        const double ln = (w + 1 < L.n_windows) ? L.lambda[w + 1] : li;
        wc.hkd = 0.5 * L.k * (ln - li);
        wc.ssum = ln + li;
        const double c = 2.0 * wc.hkd / L.kT;
        wc.ch = (float)c;
        wc.cl = (float)(c - (double)wc.ch);
        wc.li_h = (float)li;
        wc.li_m = (float)(li - (double)wc.li_h);
        wc.li_l = (float)((li - (double)wc.li_h) - (double)wc.li_m);
        wc.sgn = wc.hkd < 0 ? -1.f : 1.f;
        wc.k = exp_consts();
    }
    if (T == 0) {
        if (threadIdx.x == 0) out[(size_t)w * L.replicas + r] = Partial{INFINITY, 0.0, 0.0, 0.0, 0.0};
        return;
    }
    __syncthreads();
    // x_ref: the largest x if w falls with x (hkd > 0), else the smallest
    const float sgn = wc.sgn;
    float mx = -INFINITY;
    for (long long t = threadIdx.x; t < T; t += kPartialThreads) mx = fmaxf(mx, sgn * x[t]);
    const float xref = sgn * block_max_f<kPartialThreads>(mx, redf);
    const float ch = wc.ch, cl = wc.cl, li_h = wc.li_h, li_m = wc.li_m, li_l = wc.li_l;
    const ExpConsts k = wc.k;
    double S = 0, s1 = 0, s2 = 0;
    float Sh = 0, Sl = 0, ah1 = 0, al1 = 0, ah2 = 0, al2 = 0;
    int cnt = 0;
    for (long long t = threadIdx.x; t < T; t += kPartialThreads) {
        const float xv = x[t];
        float dh, dl;
        two_sum_f(xv, -xref, dh, dl);  // x - x_ref exactly
        float ah = ch * dh;
        float al = fmaf(ch, dh, -ah) + (ch * dl + cl * dh);
        fast_two_sum_f(ah, al, ah, al);
        float eh, el;
        exp_ff(ah, al, k, tab_hi, tab_lo, eh, el);
        ff_add(Sh, Sl, eh, el);
        // d = x - lambda_i: x - li_h exactly, then the rest of lambda_i
        float qh, ql;
        two_sum_f(xv, -li_h, qh, ql);
        ff_add(qh, ql, -li_m, -li_l);
        ff_add(ah1, al1, qh, ql);
        const float ph = qh * qh;
        const float pl = fmaf(qh, qh, -ph) + 2.f * qh * ql;
        ff_add(ah2, al2, ph, pl);
        if (++cnt == kFlushSamples) {
            S += (double)Sh + (double)Sl;
            s1 += (double)ah1 + (double)al1;
            s2 += (double)ah2 + (double)al2;
            Sh = Sl = ah1 = al1 = ah2 = al2 = 0.f;
            cnt = 0;
        }
    }
    S += (double)Sh + (double)Sl;
    s1 += (double)ah1 + (double)al1;
    s2 += (double)ah2 + (double)al2;
    const double Sb = block_sum<kPartialThreads>(S, red);
    const double sdx = block_sum<kPartialThreads>(s1, red);
    const double sdx2 = block_sum<kPartialThreads>(s2, red);
    // the minimum of w, taken at x_ref, in the FP64 form of Eq. (9)
    if (threadIdx.x == 0)
        out[(size_t)w * L.replicas + r] = Partial{wc.hkd * (wc.ssum - 2.0 * (double)xref), Sb, (double)T, sdx, sdx2};
}

constexpr int kWindowThreads = 256;

// Replica counts up to this keep the per-replica exponential sums E[r] in
// shared memory; larger ones recompute them in the jackknife loops.
constexpr int kWindowSmemReplicas = 16384;

// Error-free sum of two doubles: s + e == a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e)
{
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Block-wide sum of compensated pairs (s, c) (each thread's Neumaier sum):
// the pairs are merged with TwoSum so the result hi + lo keeps the
// compensation; hi is the correctly rounded total up to O(n eps^2).
template <int NT> __device__ void block_sum_pair(double s, double c, double *red, double &hi, double &lo)
{
    for (int o = 16; o > 0; o >>= 1) {
        const double s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
        double t, e;
        two_sum(s, s2, t, e);
        s = t;
        c = c + c2 + e;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) {
        red[2 * warp] = s;
        red[2 * warp + 1] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = red[0], tc = red[1];
        for (int q = 1; q < NT / 32; ++q) {
            double t, e;
            two_sum(ts, red[2 * q], t, e);
            ts = t;
            tc = tc + red[2 * q + 1] + e;
        }
        const double h = ts + tc;
        red[2 * (NT / 32)] = h;
        red[2 * (NT / 32) + 1] = tc - (h - ts);
    }
    __syncthreads();
    hi = red[2 * (NT / 32)];
    lo = red[2 * (NT / 32) + 1];
}

// Sum of the replicas' exponential sums without replica r, from the
// compensated total hi + lo of all of them: (hi - e_r) + lo.  The terms are
// non-negative, so the only cancellation is e_r close to the total, and then
// hi - e_r is exact (Sterbenz: e_r >= hi / 2) and the result carries the
// total's own accuracy; otherwise hi - e_r >= hi / 2 rounds once.  O(1) per
// replica instead of re-summing the other R - 1 terms.
__device__ __forceinline__ double sum_without(double hi, double lo, double e_r)
{
    const double v = (hi - e_r) + lo;
    return v > 0.0 ? v : 0.0;
}

template <bool SMEM>
__global__ void __launch_bounds__(kWindowThreads) window_kernel(const ReduceLayout L, const Partial *P, WindowOut *wo)
{
    extern __shared__ double E[];  // [replicas] when SMEM
    __shared__ double red[2 * (kWindowThreads / 32 + 1)];
    const int w = blockIdx.x, R = L.replicas;
    const Partial *p = P + (size_t)w * R;
    const double li = L.lambda[w];
    const double ln = (w + 1 < L.n_windows) ? L.lambda[w + 1] : li;
    const double d = ln - li;
    double m = INFINITY;
    for (int r = threadIdx.x; r < R; r += kWindowThreads)
        if (p[r].n > 0) m = fmin(m, p[r].m);
    m = block_min<kWindowThreads>(m, red);
    // replica r's exponential sum brought to the window's common shift m
    auto e_of = [&](int r) { return p[r].n > 0 ? p[r].S * exp(-(p[r].m - m) / L.kT) : 0.0; };
    double se = 0, ce = 0, sn = 0, s1 = 0, c1 = 0, s2 = 0, c2 = 0;
    for (int r = threadIdx.x; r < R; r += kWindowThreads) {
        const double e = e_of(r);
        if (SMEM) E[r] = e;
        neumaier(se, ce, e);
        sn += p[r].n;
        neumaier(s1, c1, p[r].sdx);
        neumaier(s2, c2, p[r].sdx2);
    }
    double Shi, Slo;
    block_sum_pair<kWindowThreads>(se, ce, red, Shi, Slo);
    const double S = Shi + Slo;
    const double n = block_sum<kWindowThreads>(sn, red);
    const double sdx = block_sum<kWindowThreads>(s1 + c1, red);
    const double sdx2 = block_sum<kWindowThreads>(s2 + c2, red);
    const double je = m - L.kT * log(S / n);
    const double mdx = sdx / n;
    const double mean = li + mdx;
    const double var = sdx2 / n - mdx * mdx;
    const double fl = -L.k * d * mdx;
    const double g2 = L.k * var / L.kT;
    // delete-one-replica jackknife, O(R): the leave-one-out exponential sum
    // from the compensated total (sum_without), the Eq. (14) mean from sdx
    double vje = 0, vfl = 0;
    const bool jk = R >= 2;
    if (jk) {
        for (int r = threadIdx.x; r < R; r += kWindowThreads) {
            const double sm = sum_without(Shi, Slo, SMEM ? E[r] : e_of(r));
            const double nm = n - p[r].n;
            vje += m - L.kT * log(sm / nm);
            vfl += -L.k * d * (sdx - p[r].sdx) / nm;
        }
    }
    const double mje = block_sum<kWindowThreads>(vje, red) / R;
    const double mfl = block_sum<kWindowThreads>(vfl, red) / R;
    double qje = 0, qfl = 0;
    if (jk) {
        for (int r = threadIdx.x; r < R; r += kWindowThreads) {
            const double sm = sum_without(Shi, Slo, SMEM ? E[r] : e_of(r));
            const double nm = n - p[r].n;
            const double a = m - L.kT * log(sm / nm) - mje;
            const double b = -L.k * d * (sdx - p[r].sdx) / nm - mfl;
            qje += a * a;
            qfl += b * b;
        }
    }
    const double sje = block_sum<kWindowThreads>(qje, red);
    const double sfl = block_sum<kWindowThreads>(qfl, red);
    if (threadIdx.x == 0) {
        WindowOut o;
        o.je = je;
        o.fl = fl;
        o.g = L.k * d * d / 2.0 * (1.0 - g2) + fl;
        o.wmean = 0.5 * L.k * d * (ln + li - 2.0 * mean);
        o.varw = L.k * L.k * d * d * var;
        o.n = n;
        o.jk_je = jk ? (R - 1.0) / R * sje : NAN;
        o.jk_fl = jk ? (R - 1.0) / R * sfl : NAN;
        o.mean = mean;
        o.var = var;
        wo[w] = o;
    }
}

// Stage 3: the profiles are prefix sums over the windows of the per-window
// increments (and a prefix minimum of the sample counts); one CTA scans them
// kProfileThreads windows at a time (warp shuffles, then the warps' totals),
// carrying the running totals from one chunk to the next, and every thread
// writes its window's fields.
constexpr int kProfileThreads = 256;
constexpr int kProfileSums = 7;  // je, fl, g, wmean, jk_je, jk_fl, varw

__global__ void __launch_bounds__(kProfileThreads) profile_kernel(const ReduceLayout L, const WindowOut *wo,
                                                                  double *out)
{
    __shared__ double wsum[kProfileThreads / 32][kProfileSums + 1];
    __shared__ double carry[kProfileSums + 1];
    const int s = L.n_windows, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid <= kProfileSums) carry[tid] = tid < kProfileSums ? 0.0 : INFINITY;
    __syncthreads();
    for (int base = 0; base < s; base += kProfileThreads) {
        const int j = base + tid;
        // window j's own terms: the increment of the pair (j - 1, j)
        double v[kProfileSums + 1];
        if (j > 0 && j < s) {
            const WindowOut &o = wo[j - 1];
            v[0] = o.je; v[1] = o.fl; v[2] = o.g; v[3] = o.wmean; v[4] = o.jk_je; v[5] = o.jk_fl; v[6] = o.varw;
            v[7] = o.n;
        } else {
            for (int q = 0; q < kProfileSums; ++q) v[q] = 0.0;
            v[kProfileSums] = INFINITY;
        }
        // inclusive scan inside the warp
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
            for (int q = 0; q <= kProfileSums; ++q) {
                const double u = __shfl_up_sync(0xffffffffu, v[q], o);
                if (lane >= o) v[q] = q < kProfileSums ? v[q] + u : fmin(v[q], u);
            }
        }
        if (lane == 31)
            for (int q = 0; q <= kProfileSums; ++q) wsum[warp][q] = v[q];
        __syncthreads();
        // add the earlier warps' totals and the carry of the earlier chunks
        double pre[kProfileSums + 1];
        for (int q = 0; q <= kProfileSums; ++q) pre[q] = carry[q];
        for (int w = 0; w < warp; ++w)
            for (int q = 0; q <= kProfileSums; ++q)
                pre[q] = q < kProfileSums ? pre[q] + wsum[w][q] : fmin(pre[q], wsum[w][q]);
        for (int q = 0; q <= kProfileSums; ++q) v[q] = q < kProfileSums ? pre[q] + v[q] : fmin(pre[q], v[q]);
        if (j < s) {
            double *f[kResFields];
            for (int q = 0; q < kResFields; ++q) f[q] = out + (size_t)q * s;
            const double je = v[0], fl = v[1], Q = v[7];
            const double lam = L.lambda[j];
            f[kResLambda][j] = lam;
            f[kResJE][j] = je;
            f[kResFluct][j] = fl;
            f[kResG][j] = v[2];
            f[kResCom][j] = 0.5 * (je + fl);
            f[kResUnc][j] = 0.5 * (je - fl);
            f[kResSeJE][j] = j > 0 ? sqrt(v[4]) : 0.0;
            f[kResSeFluct][j] = j > 0 ? sqrt(v[5]) : 0.0;
            f[kResVarZW][j] = (j > 0 && Q > 1) ? v[6] / Q + v[6] * v[6] / (2.0 * L.kT * L.kT * (Q - 1.0))
                                               : (j > 0 ? NAN : 0.0);
            f[kResWMean][j] = v[3];
            f[kResAccForce][j] = j > 0 ? fl / (lam - L.lambda[0]) : 0.0;
            f[kResMeanX][j] = wo[j].mean;
            f[kResVarX][j] = wo[j].var;
            f[kResGamma2][j] = L.k * wo[j].var / L.kT;
        }
        __syncthreads();  // every thread has read carry and wsum
        if (tid == kProfileThreads - 1)
            for (int q = 0; q <= kProfileSums; ++q) carry[q] = v[q];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Eq. (5) and Eq. (15).  The free energy of turning the trap on at lambda_1,
// dF(lambda_1, k) = kT ln < exp(u / kT) >, u = k/2 (x_1 - lambda_1)^2, over the
// first window's samples, and the state free energy
// G(lambda_j, lambda_1) = dF^JE(lambda_j, lambda_1, k) - dF(lambda_1, k).
// Stage 1 (one CTA per replica of the first window): the replica's
// max-shifted sum in the form of the JE partials with w = -u:
// m = min w = -max u, S = sum exp(-(w - m)/kT) = sum exp((u - max u)/kT).
// Stage 2 (one CTA): the turn-on estimate, G at every profile point, and the
// delete-one-replica jackknife (the first window's replica r is left out of
// its JE increment and of the turn-on average together; the other windows'
// jackknife variances of their increments are added).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kPartialThreads) turn_on_partial_kernel(const ReduceLayout L, Partial *out)
{
    __shared__ double red[kPartialThreads / 32 + 1];
    const int r = blockIdx.x;
    const long long T = L.tw[0];
    const float *x = L.x + L.off_w[0] + (long long)r * T;
    const double l1 = L.lambda[0], hk = 0.5 * L.k, beta = 1.0 / L.kT;
    double m = INFINITY, S = 0;
    for (long long t = threadIdx.x; t < T; t += kPartialThreads) {
        const double d = (double)x[t] - l1;
        const double wv = -hk * d * d;
        if (wv < m) {
            S = (m == INFINITY ? 0.0 : S * exp((wv - m) * beta)) + 1.0;
            m = wv;
        } else {
            S += exp((m - wv) * beta);
        }
    }
    const double mb = block_min<kPartialThreads>(m, red);
    const double St = m == INFINITY ? 0.0 : S * exp((mb - m) * beta);
    const double Sb = block_sum<kPartialThreads>(St, red);
    if (threadIdx.x == 0) out[r] = Partial{mb, Sb, (double)T, 0.0, 0.0};
}

// The window's exponential sums of the replicas on a common shift: the
// shift (minimum of the replicas' minima) and the compensated total.
template <int NT>
__device__ void common_shift_sum(const Partial *p, int R, double kT, double *red, double &m, double &hi, double &lo,
                                 double &n)
{
    double mm = INFINITY;
    for (int r = threadIdx.x; r < R; r += NT)
        if (p[r].n > 0) mm = fmin(mm, p[r].m);
    m = block_min<NT>(mm, red);
    double se = 0, ce = 0, sn = 0;
    for (int r = threadIdx.x; r < R; r += NT) {
        neumaier(se, ce, p[r].n > 0 ? p[r].S * exp(-(p[r].m - m) / kT) : 0.0);
        sn += p[r].n;
    }
    block_sum_pair<NT>(se, ce, red, hi, lo);
    n = block_sum<NT>(sn, red);
}

__global__ void __launch_bounds__(kWindowThreads) state_kernel(const ReduceLayout L, const Partial *P, const Partial *Pt,
                                                               const WindowOut *wo, double *out)
{
    __shared__ double red[2 * (kWindowThreads / 32 + 1)];
    const int R = L.replicas, s = L.n_windows;
    const double kT = L.kT;
    double m0, S0h, S0l, n, mt, Sth, Stl, nt;
    common_shift_sum<kWindowThreads>(P, R, kT, red, m0, S0h, S0l, n);   // first window, Eq. (12)
    common_shift_sum<kWindowThreads>(Pt, R, kT, red, mt, Sth, Stl, nt);  // first window, Eq. (5)
    const double on = kT * log((Sth + Stl) / nt) - mt;
    // leave-one-out values of the first window: its JE increment minus the
    // turn-on estimate (g), and the turn-on estimate alone (t)
    auto e_of = [&](const Partial &q, double mm) { return q.n > 0 ? q.S * exp(-(q.m - mm) / kT) : 0.0; };
    double vg = 0, vt = 0;
    const bool jk = R >= 2;
    if (jk) {
        for (int r = threadIdx.x; r < R; r += kWindowThreads) {
            const double nm = n - P[r].n;
            const double t = kT * log(sum_without(Sth, Stl, e_of(Pt[r], mt)) / nm) - mt;
            const double je = m0 - kT * log(sum_without(S0h, S0l, e_of(P[r], m0)) / nm);
            vg += je - t;
            vt += t;
        }
    }
    const double mg = block_sum<kWindowThreads>(vg, red) / R;
    const double mtt = block_sum<kWindowThreads>(vt, red) / R;
    double qg = 0, qt = 0;
    if (jk) {
        for (int r = threadIdx.x; r < R; r += kWindowThreads) {
            const double nm = n - P[r].n;
            const double t = kT * log(sum_without(Sth, Stl, e_of(Pt[r], mt)) / nm) - mt;
            const double je = m0 - kT * log(sum_without(S0h, S0l, e_of(P[r], m0)) / nm);
            qg += (je - t - mg) * (je - t - mg);
            qt += (t - mtt) * (t - mtt);
        }
    }
    const double var_g = (R - 1.0) / R * block_sum<kWindowThreads>(qg, red);
    const double var_t = (R - 1.0) / R * block_sum<kWindowThreads>(qt, red);
    if (threadIdx.x == 0) {
        double je = 0, v = var_g;
        for (int j = 0; j < s; ++j) {
            if (j > 0) je += wo[j - 1].je;
            if (j > 1) v += wo[j - 1].jk_je;
            out[j] = je - on;                                              // G(lambda_j, lambda_1)
            out[s + j] = jk ? sqrt(j == 0 ? var_t : v) : NAN;              // its standard error
        }
        out[2 * s] = on;                                                   // dF(lambda_1, k), Eq. (5)
    }
}

cudaError_t state_launch(const ReduceLayout &L, void *scratch, void *turn_partials, double *out, cudaStream_t st)
{
    const Partial *P = static_cast<const Partial *>(scratch);
    const WindowOut *wo =
        reinterpret_cast<const WindowOut *>(static_cast<const char *>(scratch) + partial_bytes(L.n_windows, L.replicas));
    Partial *Pt = static_cast<Partial *>(turn_partials);
    turn_on_partial_kernel<<<L.replicas, kPartialThreads, 0, st>>>(L, Pt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    state_kernel<<<1, kWindowThreads, 0, st>>>(L, P, Pt, wo, out);
    return cudaGetLastError();
}

size_t reduce_scratch_bytes(int n_windows, int replicas)
{
    return sizeof(Partial) * (size_t)n_windows * replicas + sizeof(WindowOut) * (size_t)n_windows + 256;
}

cudaError_t partials_launch(const ReduceLayout &L, void *P, cudaStream_t st)
{
    partial_kernel<<<dim3(L.n_windows, L.replicas), kPartialThreads, 0, st>>>(L, static_cast<Partial *>(P));
    return cudaGetLastError();
}

cudaError_t combine_launch(const ReduceLayout &L, const void *P, void *window_scratch, double *out, cudaStream_t st)
{
    const Partial *pp = static_cast<const Partial *>(P);
    WindowOut *wo = static_cast<WindowOut *>(window_scratch);
    cudaError_t e;
    if (L.replicas <= kWindowSmemReplicas) {
        const size_t smem = sizeof(double) * (size_t)L.replicas;
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(window_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        window_kernel<true><<<L.n_windows, kWindowThreads, smem, st>>>(L, pp, wo);
    } else {
        window_kernel<false><<<L.n_windows, kWindowThreads, 0, st>>>(L, pp, wo);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    profile_kernel<<<1, kProfileThreads, 0, st>>>(L, wo, out);
    return cudaGetLastError();
}

// Constant-velocity pulling, record j (one block each): over the replicas,
// the Jarzynski average of the accumulated work, its mean and variance (the
// second-order cumulant estimate) and the mean reaction coordinate.
__global__ void __launch_bounds__(kWindowThreads) smd_stats_kernel(const double *W, const float *x, int R, long long T,
                                                                   double kT, double *out)
{
    __shared__ double red[kWindowThreads / 32 + 1];
    const long long j = blockIdx.x;
    double m = INFINITY;
    for (int r = threadIdx.x; r < R; r += kWindowThreads) m = fmin(m, W[(size_t)r * T + j]);
    m = block_min<kWindowThreads>(m, red);
    double se = 0, ce = 0, sw = 0, cw = 0, sx = 0, cx = 0;
    for (int r = threadIdx.x; r < R; r += kWindowThreads) {
        const double w = W[(size_t)r * T + j];
        neumaier(se, ce, exp(-(w - m) / kT));
        neumaier(sw, cw, w);
        neumaier(sx, cx, (double)x[(size_t)r * T + j]);
    }
    const double S = block_sum<kWindowThreads>(se + ce, red);
    const double mean = block_sum<kWindowThreads>(sw + cw, red) / R;
    const double mx = block_sum<kWindowThreads>(sx + cx, red) / R;
    double sv = 0, cv = 0;
    for (int r = threadIdx.x; r < R; r += kWindowThreads) {
        const double d = W[(size_t)r * T + j] - mean;
        neumaier(sv, cv, d * d);
    }
    const double var = block_sum<kWindowThreads>(sv + cv, red) / R;
    if (threadIdx.x == 0) {
        out[0 * T + j] = m - kT * log(S / R);
        out[1 * T + j] = mean - var / (2.0 * kT);
        out[2 * T + j] = mean;
        out[3 * T + j] = var;
        out[4 * T + j] = mx;
    }
}

cudaError_t smd_stats_launch(const double *W, const float *x, int R, long long T, double kT, double *out,
                             cudaStream_t st)
{
    if (T < 1) return cudaSuccess;
    smd_stats_kernel<<<(unsigned)T, kWindowThreads, 0, st>>>(W, x, R, T, kT, out);
    return cudaGetLastError();
}

size_t partial_bytes(int n_windows, int replicas) { return sizeof(Partial) * (size_t)n_windows * replicas; }

cudaError_t reduce_launch(const ReduceLayout &L, void *scratch, double *out, cudaStream_t st)
{
    void *P = scratch;
    void *wo = static_cast<char *>(scratch) + partial_bytes(L.n_windows, L.replicas);
    cudaError_t e = partials_launch(L, P, st);
    if (e != cudaSuccess) return e;
    return combine_launch(L, P, wo, out, st);
}

__global__ void work_increment_kernel(const ReduceLayout L, double *out)
{
    const int w = blockIdx.y, r = blockIdx.z;
    const long long T = L.tw[w];
    const double li = L.lambda[w], ln = L.lambda[w + 1];
    const double hkd = 0.5 * L.k * (ln - li), ssum = ln + li;
    const long long base = L.off_w[w] + (long long)r * T;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < T; t += (long long)gridDim.x * blockDim.x)
        out[base + t] = hkd * (ssum - 2.0 * (double)L.x[base + t]);
}

__global__ void work_paired_kernel(const ReduceLayout L, long long T, double *out)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long n = (long long)L.replicas * T;
    if (idx >= n) return;
    double W = 0.0;
    for (int i = 0; i + 1 < L.n_windows; ++i) {
        const double li = L.lambda[i], ln = L.lambda[i + 1];
        W += 0.5 * L.k * (ln - li) * (ln + li - 2.0 * (double)L.x[L.off_w[i] + idx]);
        out[(size_t)i * n + idx] = W;
    }
}

cudaError_t work_samples_launch(const ReduceLayout &L, int mode, long long samples_per_replica, double *out,
                                cudaStream_t st)
{
    if (mode == 0) {
        const int bx = (int)((samples_per_replica + 255) / 256 > 64 ? 64 : (samples_per_replica + 255) / 256);
        work_increment_kernel<<<dim3(bx > 0 ? bx : 1, L.n_windows - 1, L.replicas), 256, 0, st>>>(L, out);
    } else {
        const long long n = (long long)L.replicas * samples_per_replica;
        work_paired_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(L, samples_per_replica, out);
    }
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Allocation-free variant of the reduction (pmf_free_energy_noalloc).
//
// Its scratch (replica partials, window results, sample offsets) lives in one
// file-scope device array of fixed size instead of memory obtained from
// cudaMalloc.  Every GPU that loads the library holds this array until the
// process exits, and every call on that GPU reuses it: two calls whose work
// overlaps on the GPU (different streams, or a second call before the first
// has finished) write the same scratch and race.  Nothing in it has to start
// at zero: each call rewrites every entry it later reads.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kNoAllocPartialBytes = sizeof(Partial) * (size_t)kNoAllocMaxWindowReplicas;
constexpr size_t kNoAllocWindowBytes = sizeof(WindowOut) * (size_t)kNoAllocMaxWindows;
constexpr size_t kNoAllocLayoutBytes = 2 * sizeof(long long) * (size_t)kNoAllocMaxWindows;
constexpr size_t kNoAllocBytes = kNoAllocPartialBytes + kNoAllocWindowBytes + kNoAllocLayoutBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Host side: the array's name is only a host stand-in; its device address is
// looked up with that device current and cached per device, together with
// the unique id of the CUDA context it was looked up in.  A later call in
// another context of the same device (after cudaDeviceReset, the module and
// its array are loaded again, maybe elsewhere) looks the address up again.
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_addr[kMaxDevices] = {};
unsigned long long g_noalloc_ctx[kMaxDevices] = {};

// Unique id of the calling thread's current context (driver entry points
// cuCtxGetCurrent / cuCtxGetId, reached through the runtime so the library
// links no driver library); 0 if it cannot be had.
unsigned long long current_context_id()
{
    using GetCurrent = int (*)(void **);
    using GetId = int (*)(void *, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == 0 && ctx && get_id(ctx, &id) == 0) return id;
    return 0;
}

cudaError_t noalloc_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    const unsigned long long ctx = current_context_id();
    if (g_noalloc_addr[dev] == nullptr || ctx == 0 || ctx != g_noalloc_ctx[dev]) {
        // (the lookup makes the device's primary context current if no
        // runtime call has done so yet; the id is read again after it)
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
        g_noalloc_ctx[dev] = current_context_id();
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

__global__ void noalloc_layout_kernel(long long *off, long long *tw, int n_windows, int replicas, long long T)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_windows) {
        off[i] = (long long)i * replicas * T;
        tw[i] = T;
    }
}

}  // namespace

cudaError_t reduce_noalloc_launch(const float *x, const double *lambda, int n_windows, int replicas,
                                  long long samples_per_window, double k, double kT, double *out, cudaStream_t st)
{
    void *base = nullptr;
    cudaError_t e = noalloc_scratch(&base);
    if (e != cudaSuccess) return e;
    unsigned char *b = static_cast<unsigned char *>(base);
    long long *off = reinterpret_cast<long long *>(b + kNoAllocPartialBytes + kNoAllocWindowBytes);
    long long *tw = off + kNoAllocMaxWindows;
    noalloc_layout_kernel<<<(n_windows + 127) / 128, 128, 0, st>>>(off, tw, n_windows, replicas, samples_per_window);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    Partial *P = reinterpret_cast<Partial *>(b);
    WindowOut *wo = reinterpret_cast<WindowOut *>(b + kNoAllocPartialBytes);
    ReduceLayout L;
    L.x = x;
    L.lambda = lambda;
    L.off_w = off;
    L.tw = tw;
    L.n_windows = n_windows;
    L.replicas = replicas;
    L.k = k;
    L.kT = kT;
    if ((e = partials_launch(L, P, st)) != cudaSuccess) return e;
    return combine_launch(L, P, wo, out, st);
}

}  // namespace pmf
