// Surrogate MLP lambda -> (mu, log sigma^2) of the reaction coordinate,
// trained on the windows' own x samples (the learned window-placement part).
//
// Network 1 -> 64 -> 64 -> 2 with SiLU; Gaussian negative log-likelihood
// 0.5 [s + (x' - mu')^2 e^{-s}] in normalised units lambda' = (lambda - c)/h,
// x' = (x - c)/h; Adam on FP32 master weights.
//
// One CTA of 128 threads (one warpgroup); thread t owns sample t of a
// 128-sample tile.  The 64x64 layer runs on the 5th-generation tensor cores:
// BF16 operands staged in shared memory in the K-major no-swizzle core-matrix
// layout, tcgen05.mma issued by one thread with FP32 accumulators in tensor
// memory, completion through tcgen05.commit on an mbarrier, results read back
// with tcgen05.ld.  Three products per tile:
//   Z2   = H1 W2^T            (M 128 samples, N 64, K 64)
//   dH1  = dZ2 W2             (M 128 samples, N 64, K 64; B = W2^T staged)
//   dW2 += dZ2^T H1           (M 128 (rows 64..127 zero), N 64, K 128 samples)
// Layers 1 and 3, SiLU and the loss run on the FP32 ALUs.
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"
#include "internal.h"

namespace pmf {

namespace {

constexpr int kH = 64;
constexpr int kTile = kMlpTile;
// parameter offsets in the packed FP32 vector
constexpr int oW1 = 0, oB1 = 64, oW2 = 128, oB2 = 128 + 4096, oW3 = oB2 + 64, oB3 = oW3 + 128;
static_assert(oB3 + 2 == kMlpParams, "parameter packing");

// ---- shared-memory tile layout for tcgen05 (K-major, no swizzle) --------
// element (row r, k) of a tile with K columns lives at byte
//   (r / 8) * SBO + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,  SBO = K / 8 * 128,
// i.e. 8x8 core matrices (8 rows of 16 bytes), the K direction first.
__device__ __forceinline__ uint32_t core_offset(int r, int k, int K)
{
    return (uint32_t)((r >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start >> 4 in bits 0-13, leading byte
// offset (K direction, between core matrices) >> 4 in bits 16-29, stride
// byte offset (M/N direction, between 8-row groups) >> 4 in bits 32-45,
// descriptor version 1 in bits 46-47, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdescM128N64 = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdescM128N64), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
                 : "memory");
}

// Bounded wait on an mbarrier phase; returns false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t phase)
{
    const uint32_t a = smem_addr(mbar);
    for (int it = 0; it < (1 << 26); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z)
{
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

__device__ __forceinline__ void put_bf16(unsigned char *tile, uint32_t off, float v)
{
    *reinterpret_cast<__nv_bfloat16 *>(tile + off) = __float2bfloat16_rn(v);
}

struct MlpSmem {
    unsigned char *aH1;    // [128 x 64]  H1 (A of Z2, sample-major)
    unsigned char *aDZ2;   // [128 x 64]  dZ2 (A of dH1)
    unsigned char *bW2;    // [64 x 64]   W2 (B of Z2: n = out, k = in)
    unsigned char *bW2T;   // [64 x 64]   W2^T (B of dH1: n = in, k = out)
    unsigned char *aDZ2T;  // [128 x 128] dZ2^T, rows 64..127 zero (A of dW2, k = sample)
    unsigned char *bH1T;   // [64 x 128]  H1^T (B of dW2: n = in, k = sample)
    float *h2;             // [128][65]   fp32 H2, then dZ1
    float *dz2;            // [128][65]   fp32 dZ2
    float *dout;           // [128][2]
    float *lam;            // [128]
    float *w;              // [kMlpParams] fp32 weights
    float *grad;           // [kMlpParams] gradient accumulators
    uint64_t *mbar;
    uint32_t *tmem_slot;
    float *red;            // [8]
    long long *win_off;    // [kMaxSmemWindows] first sample of each window (training)
};

constexpr int kLd = 65;  // padded row length of the fp32 staging arrays
constexpr int kMaxSmemWindows = 1024;  // window offsets kept in shared memory up to this count
constexpr size_t kSmemTiles = 16384 * 2 + 8192 * 2 + 32768 + 16384;
constexpr size_t kSmemBytes = kSmemTiles + 2 * sizeof(float) * kTile * kLd + sizeof(float) * (kTile * 2 + kTile) +
                              2 * sizeof(float) * kMlpParams + 64 + 1024 + sizeof(long long) * kMaxSmemWindows;

struct MlpArgs {
    float *params;              // [kMlpParams] fp32 master weights (in/out)
    float *adam_m, *adam_v;     // [kMlpParams]
    int adam_t;                 // steps taken so far
    float lr;
    double c, h;                // normalisation lambda' = (lambda - c) / h
    // data: either explicit samples or a run's sample store
    const double *lam_in;       // [n] (explicit mode)
    const float *x_in;          // [n] (explicit mode, may be null for forward)
    int n;
    const float *xs;            // run sample store
    const double *win_lambda;   // [n_windows]
    const long long *win_off;   // [n_windows]
    const long long *win_tw;    // [n_windows]
    int n_windows, replicas;
    long long total;
    int mode;                   // 0 forward, 1 gradient, 2 train, 3 one tile of a training step
    int steps, batch;
    unsigned long long seed;
    double *out_mu, *out_logvar;  // forward outputs [n]
    float *out_grad;            // gradient mode [kMlpParams]
    double *out_loss;           // gradient / train: last batch loss
    float *tile_grad;           // mode 3: [tiles][kMlpParams] gradient of each CTA's tile
    double *tile_loss;          // mode 3: [tiles] loss sum of each CTA's tile
    int *err;
};

__device__ void stage_w2(const MlpSmem &s)
{
    for (int e = threadIdx.x; e < kH * kH; e += kTile) {
        const int o = e >> 6, i = e & 63;
        const float w = s.w[oW2 + e];
        put_bf16(s.bW2, core_offset(o, i, 64), w);
        put_bf16(s.bW2T, core_offset(i, o, 64), w);
    }
}

// One tile of up to 128 samples: forward, and (grad) backward into s.grad.
// Returns false on an mbarrier timeout.
__device__ bool mlp_tile(const MlpArgs &a, const MlpSmem &s, uint32_t tmem, uint32_t &phase, int count, float inv_batch,
                         bool grad, bool first_tile, double *loss_acc)
{
    const int t = threadIdx.x, warp = t >> 5;
    const bool live = t < count;
    const float lam = s.lam[t];
    // layer 1 (fp32) -> H1 as bf16 in both layouts
#pragma unroll 8
    for (int f = 0; f < kH; ++f) {
        const float z1 = fmaf(s.w[oW1 + f], lam, s.w[oB1 + f]);
        const float h1 = live ? silu(z1) : 0.f;
        put_bf16(s.aH1, core_offset(t, f, 64), h1);
        put_bf16(s.bH1T, core_offset(f, t, 128), h1);
    }
    fence_async_smem();
    __syncthreads();
    if (t == 0) {
        tc_after_sync();
#pragma unroll
        for (int k = 0; k < 4; ++k)
            mma_bf16(tmem + 0, smem_desc(smem_addr(s.aH1) + 256 * k, 128, 1024),
                     smem_desc(smem_addr(s.bW2) + 256 * k, 128, 1024), k > 0);
        mma_commit(s.mbar);
    }
    if (!mbar_wait(s.mbar, phase)) return false;
    phase ^= 1u;
    tc_after_sync();
    // H2 = silu(Z2 + b2), out = W3 H2 + b3
    float mu = s.w[oB3 + 0], lv = s.w[oB3 + 1];
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float z[16];
        tmem_ld16(lane_base + 0 + 16 * c, z);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int f = 16 * c + q;
            const float z2 = z[q] + s.w[oB2 + f];
            const float h2 = silu(z2);
            s.h2[t * kLd + f] = z2;  // keep Z2 for the backward pass
            mu = fmaf(s.w[oW3 + f], h2, mu);
            lv = fmaf(s.w[oW3 + 64 + f], h2, lv);
        }
    }
    if (!grad) {
        s.dout[2 * t] = mu;
        s.dout[2 * t + 1] = lv;
        tc_before_sync();
        __syncthreads();
        return true;
    }
    // loss gradient (normalised units), dH2 = dout W3, dZ2 = dH2 silu'(Z2)
    const float xv = live ? s.dout[2 * t] : 0.f;  // x' staged by the caller in dout[2t]
    const float e = __expf(-lv);
    const float r = xv - mu;
    const float dmu = live ? -r * e * inv_batch : 0.f;
    const float dlv = live ? 0.5f * (1.f - r * r * e) * inv_batch : 0.f;
    {  // loss: one shared-memory atomic per warp instead of one per sample
        float lo = live ? 0.5f * (lv + r * r * e) : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lo += __shfl_xor_sync(0xffffffffu, lo, o);
        if ((t & 31) == 0) atomicAdd(loss_acc, (double)lo);
    }
    s.dout[2 * t] = dmu;
    s.dout[2 * t + 1] = dlv;
#pragma unroll 8
    for (int f = 0; f < kH; ++f) {
        const float z2 = s.h2[t * kLd + f];
        const float dh2 = fmaf(dmu, s.w[oW3 + f], dlv * s.w[oW3 + 64 + f]);
        const float d = live ? dh2 * silu_grad(z2) : 0.f;
        s.dz2[t * kLd + f] = d;
        s.h2[t * kLd + f] = silu(z2);  // H2 for dW3
        put_bf16(s.aDZ2, core_offset(t, f, 64), d);
        put_bf16(s.aDZ2T, core_offset(f, t, 128), d);
    }
    if (first_tile) {  // rows 64..127 of the dW2 A operand stay zero
        for (int e2 = t; e2 < 64 * 128; e2 += kTile) put_bf16(s.aDZ2T, core_offset(64 + (e2 >> 7), e2 & 127, 128), 0.f);
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    if (t == 0) {
        tc_after_sync();
#pragma unroll
        for (int k = 0; k < 4; ++k)
            mma_bf16(tmem + 64, smem_desc(smem_addr(s.aDZ2) + 256 * k, 128, 1024),
                     smem_desc(smem_addr(s.bW2T) + 256 * k, 128, 1024), k > 0);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            mma_bf16(tmem + 128, smem_desc(smem_addr(s.aDZ2T) + 256 * k, 128, 2048),
                     smem_desc(smem_addr(s.bH1T) + 256 * k, 128, 2048), (k > 0 || !first_tile) ? 1u : 0u);
        mma_commit(s.mbar);
    }
    // meanwhile: dW3, db3 and db2 by feature threads
    // (sums over the tile's samples in four interleaved partial sums, so
    // consecutive additions do not wait on one another)
    for (int j = t; j < 2 * kH + 2 + kH; j += kTile) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        if (j < 2 * kH) {
            const int o = j >> 6, f = j & 63;
#pragma unroll 4
            for (int q = 0; q < kTile; ++q) acc[q & 3] = fmaf(s.dout[2 * q + o], s.h2[q * kLd + f], acc[q & 3]);
            s.grad[oW3 + j] += (acc[0] + acc[1]) + (acc[2] + acc[3]);
        } else if (j < 2 * kH + 2) {
            const int o = j - 2 * kH;
#pragma unroll 4
            for (int q = 0; q < kTile; ++q) acc[q & 3] += s.dout[2 * q + o];
            s.grad[oB3 + o] += (acc[0] + acc[1]) + (acc[2] + acc[3]);
        } else {
            const int f = j - 2 * kH - 2;
#pragma unroll 4
            for (int q = 0; q < kTile; ++q) acc[q & 3] += s.dz2[q * kLd + f];
            s.grad[oB2 + f] += (acc[0] + acc[1]) + (acc[2] + acc[3]);
        }
    }
    if (!mbar_wait(s.mbar, phase)) return false;
    phase ^= 1u;
    __syncthreads();  // every thread is done reading H2 rows before they become dZ1
    tc_after_sync();
    // dZ1 = dH1 silu'(Z1)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float d[16];
        tmem_ld16(lane_base + 64 + 16 * c, d);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int f = 16 * c + q;
            const float z1 = fmaf(s.w[oW1 + f], lam, s.w[oB1 + f]);
            s.h2[t * kLd + f] = live ? d[q] * silu_grad(z1) : 0.f;  // reuse as dZ1
        }
    }
    tc_before_sync();
    __syncthreads();
    for (int j = t; j < 2 * kH; j += kTile) {
        const int f = j & 63;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        if (j < kH) {
#pragma unroll 4
            for (int q = 0; q < kTile; ++q) acc[q & 3] = fmaf(s.h2[q * kLd + f], s.lam[q], acc[q & 3]);
            s.grad[oW1 + f] += (acc[0] + acc[1]) + (acc[2] + acc[3]);
        } else {
#pragma unroll 4
            for (int q = 0; q < kTile; ++q) acc[q & 3] += s.h2[q * kLd + f];
            s.grad[oB1 + f] += (acc[0] + acc[1]) + (acc[2] + acc[3]);
        }
    }
    __syncthreads();
    return true;
}

// dW2 from tensor memory (rows 0..63 = warps 0, 1) into s.grad.
__device__ void collect_dw2(const MlpSmem &s, uint32_t tmem)
{
    const int t = threadIdx.x, warp = t >> 5;
    tc_after_sync();
    if (warp < 2) {
        const uint32_t base = tmem + ((uint32_t)(32 * warp) << 16) + 128;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float v[16];
            tmem_ld16(base + 16 * c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) s.grad[oW2 + t * 64 + 16 * c + q] += v[q];
        }
    } else {
        // the other warps take part in no tcgen05.ld; keep the sync.aligned
        // loads warp-uniform by skipping them entirely
    }
    tc_before_sync();
    __syncthreads();
}

__device__ __forceinline__ long long pick_sample(unsigned long long seed, int step, int j, long long total)
{
    const Ctr4 b = philox4x32_10(Ctr4{(uint32_t)j, (uint32_t)step, 0u, kTagMlp}, (uint32_t)seed, (uint32_t)(seed >> 32));
    const unsigned long long r = ((unsigned long long)b.b << 32) | b.a;
    return (long long)(r % (unsigned long long)total);
}

__global__ void __launch_bounds__(kTile, 1) mlp_kernel(const MlpArgs a)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    MlpSmem s;
    unsigned char *p = sm;
    s.aH1 = p; p += 16384;
    s.aDZ2 = p; p += 16384;
    s.bW2 = p; p += 8192;
    s.bW2T = p; p += 8192;
    s.aDZ2T = p; p += 32768;
    s.bH1T = p; p += 16384;
    s.h2 = reinterpret_cast<float *>(p); p += sizeof(float) * kTile * kLd;
    s.dz2 = reinterpret_cast<float *>(p); p += sizeof(float) * kTile * kLd;
    s.dout = reinterpret_cast<float *>(p); p += sizeof(float) * kTile * 2;
    s.lam = reinterpret_cast<float *>(p); p += sizeof(float) * kTile;
    s.w = reinterpret_cast<float *>(p); p += sizeof(float) * kMlpParams;
    s.grad = reinterpret_cast<float *>(p); p += sizeof(float) * kMlpParams;
    p = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
    s.mbar = reinterpret_cast<uint64_t *>(p); p += 16;
    s.tmem_slot = reinterpret_cast<uint32_t *>(p); p += 16;
    s.win_off = reinterpret_cast<long long *>(p); p += sizeof(long long) * kMaxSmemWindows;
    __shared__ double loss_acc;

    const int t = threadIdx.x, warp = t >> 5;
    // a split training step after a failed one does nothing (the host has
    // queued every step's launches; the failure is already flagged)
    if (a.mode == 3 && *(volatile int *)a.err) return;
    for (int e = t; e < kMlpParams; e += kTile) s.w[e] = a.params[e];
    if ((a.mode == 2 || a.mode == 3) && a.n_windows <= kMaxSmemWindows)
        for (int e = t; e < a.n_windows; e += kTile) s.win_off[e] = a.win_off[e];
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(s.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        loss_acc = 0.0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_addr(s.tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *s.tmem_slot;
    uint32_t phase = 0;
    bool ok = true;
    stage_w2(s);
    const float ih = (float)(1.0 / a.h);

    if (a.mode == 0 || a.mode == 1) {
        // explicit samples, tiles of 128
        for (int e = t; e < kMlpParams; e += kTile) s.grad[e] = 0.f;
        const float inv_batch = 1.f / (float)a.n;
        for (int base = 0; base < a.n && ok; base += kTile) {
            const int count = min(kTile, a.n - base);
            __syncthreads();
            const bool live = t < count;
            s.lam[t] = live ? (float)((a.lam_in[base + t] - a.c) * ih) : 0.f;
            if (a.mode == 1) s.dout[2 * t] = live ? (float)(((double)a.x_in[base + t] - a.c) * ih) : 0.f;
            __syncthreads();
            ok = mlp_tile(a, s, tmem, phase, count, inv_batch, a.mode == 1, base == 0, &loss_acc);
            if (ok && a.mode == 0 && live) {
                a.out_mu[base + t] = a.c + a.h * (double)s.dout[2 * t];
                a.out_logvar[base + t] = (double)s.dout[2 * t + 1] + 2.0 * log(a.h);
            }
        }
        if (ok && a.mode == 1) {
            collect_dw2(s, tmem);
            for (int e = t; e < kMlpParams; e += kTile) a.out_grad[e] = s.grad[e];
            if (t == 0 && a.out_loss) *a.out_loss = loss_acc / a.n;
        }
    } else if (a.mode == 3) {
        // one 128-sample tile of Adam step adam_t per CTA (tile = blockIdx.x
        // of gridDim.x): the same mini-batch draw as the one-CTA training,
        // its gradient and loss sum to this tile's slot; adam_kernel then
        // sums the tiles in a fixed order and updates the weights
        const int tile = blockIdx.x;
        const float inv_batch = 1.f / (float)(gridDim.x * kTile);
        for (int e = t; e < kMlpParams; e += kTile) s.grad[e] = 0.f;
        if (t == 0) loss_acc = 0.0;
        __syncthreads();
        const long long idx = pick_sample(a.seed, a.adam_t, tile * kTile + t, a.total);
        const long long *off = a.n_windows <= kMaxSmemWindows ? s.win_off : a.win_off;
        int lo = 0, hi = a.n_windows - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= idx) lo = mid;
            else hi = mid - 1;
        }
        s.lam[t] = (float)((a.win_lambda[lo] - a.c) * ih);
        s.dout[2 * t] = (float)(((double)a.xs[idx] - a.c) * ih);
        __syncthreads();
        ok = mlp_tile(a, s, tmem, phase, kTile, inv_batch, true, true, &loss_acc);
        if (ok) {
            collect_dw2(s, tmem);
            for (int e = t; e < kMlpParams; e += kTile) a.tile_grad[(size_t)tile * kMlpParams + e] = s.grad[e];
            if (t == 0) a.tile_loss[tile] = loss_acc;
        }
    } else {
        // training: Adam steps on mini-batches drawn from the run's samples
        const int tiles = (a.batch + kTile - 1) / kTile;
        const float inv_batch = 1.f / (float)(tiles * kTile);
        for (int step = 0; step < a.steps && ok; ++step) {
            for (int e = t; e < kMlpParams; e += kTile) s.grad[e] = 0.f;
            if (t == 0) loss_acc = 0.0;
            for (int tile = 0; tile < tiles && ok; ++tile) {
                __syncthreads();
                const long long idx = pick_sample(a.seed, a.adam_t + step, tile * kTile + t, a.total);
                // window of the sample: the last offset <= idx (bisection)
                const long long *off = a.n_windows <= kMaxSmemWindows ? s.win_off : a.win_off;
                int lo = 0, hi = a.n_windows - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (off[mid] <= idx) lo = mid;
                    else hi = mid - 1;
                }
                const int w = lo;
                s.lam[t] = (float)((a.win_lambda[w] - a.c) * ih);
                s.dout[2 * t] = (float)(((double)a.xs[idx] - a.c) * ih);
                __syncthreads();
                ok = mlp_tile(a, s, tmem, phase, kTile, inv_batch, true, tile == 0, &loss_acc);
            }
            if (!ok) break;
            collect_dw2(s, tmem);
            // Adam (Kingma & Ba) with bias correction on the fp32 masters
            const int tt = a.adam_t + step + 1;
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.f - powf(b1, (float)tt), c2 = 1.f - powf(b2, (float)tt);
#pragma unroll 8
            for (int e = t; e < kMlpParams; e += kTile) {
                const float g = s.grad[e];
                const float m = b1 * a.adam_m[e] + (1.f - b1) * g;
                const float v = b2 * a.adam_v[e] + (1.f - b2) * g * g;
                a.adam_m[e] = m;
                a.adam_v[e] = v;
                s.w[e] -= a.lr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
            }
            __syncthreads();
            stage_w2(s);
        }
        if (ok) {
            for (int e = t; e < kMlpParams; e += kTile) a.params[e] = s.w[e];
            if (t == 0 && a.out_loss) *a.out_loss = loss_acc / (tiles * kTile);
        }
    }
    if (!ok && t == 0) atomicOr(a.err, kErrTimeout);
    tc_before_sync();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

// The update half of a split training step: the tiles' gradients summed in
// tile order, then Adam (Kingma & Ba) with bias correction for step tt on
// the FP32 master weights in global memory; the last step also writes the
// batch loss.  Skipped after a failed tile launch.
__global__ void adam_kernel(float *params, float *adam_m, float *adam_v, const float *tile_grad,
                            const double *tile_loss, int tiles, int tt, float lr, double *out_loss, const int *err)
{
    if (*(const volatile int *)err) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < kMlpParams) {
        float g = 0.f;
        for (int b = 0; b < tiles; ++b) g += tile_grad[(size_t)b * kMlpParams + e];
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)tt), c2 = 1.f - powf(b2, (float)tt);
        const float m = b1 * adam_m[e] + (1.f - b1) * g;
        const float v = b2 * adam_v[e] + (1.f - b2) * g * g;
        adam_m[e] = m;
        adam_v[e] = v;
        params[e] -= lr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
    }
    if (out_loss && e == 0) {
        double l = 0.0;
        for (int b = 0; b < tiles; ++b) l += tile_loss[b];
        *out_loss = l / (double)(tiles * kTile);
    }
}

}  // namespace

cudaError_t mlp_launch(const MlpLaunch &L, cudaStream_t st)
{
    MlpArgs a{};
    a.params = L.params;
    a.adam_m = L.adam_m;
    a.adam_v = L.adam_v;
    a.adam_t = L.adam_t;
    a.lr = (float)L.lr;
    a.c = L.c;
    a.h = L.h;
    a.lam_in = L.lam_in;
    a.x_in = L.x_in;
    a.n = L.n;
    a.xs = L.xs;
    a.win_lambda = L.win_lambda;
    a.win_off = L.win_off;
    a.win_tw = L.win_tw;
    a.n_windows = L.n_windows;
    a.replicas = L.replicas;
    a.total = L.total;
    a.mode = L.mode;
    a.steps = L.steps;
    a.batch = L.batch;
    a.seed = L.seed;
    a.out_mu = L.out_mu;
    a.out_logvar = L.out_logvar;
    a.out_grad = L.out_grad;
    a.out_loss = L.out_loss;
    a.tile_grad = L.tile_grad;
    a.tile_loss = L.tile_loss;
    a.err = L.err;
    cudaError_t e = cudaFuncSetAttribute(mlp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    const int tiles = (L.batch + kTile - 1) / kTile;
    if (L.mode == 2 && L.split && tiles >= 2) {
        // one CTA per tile: per step a tile launch and an update launch
        if (!L.tile_grad || !L.tile_loss || tiles > L.tile_cap) return cudaErrorInvalidValue;
        a.mode = 3;
        for (int step = 0; step < L.steps; ++step) {
            a.adam_t = L.adam_t + step;
            mlp_kernel<<<tiles, kTile, kSmemBytes, st>>>(a);
            adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(L.params, L.adam_m, L.adam_v, L.tile_grad,
                                                                  L.tile_loss, tiles, L.adam_t + step + 1,
                                                                  (float)L.lr,
                                                                  step + 1 == L.steps ? L.out_loss : nullptr, L.err);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    mlp_kernel<<<1, kTile, kSmemBytes, st>>>(a);
    return cudaGetLastError();
}

}  // namespace pmf
