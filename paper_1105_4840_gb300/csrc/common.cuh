// Shared device helpers of libpmf (CUDA, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pmf {

// ---------------------------------------------------------------------------
// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11):
// ten rounds of two 32x32->64-bit multiplications whose high halves are
// xor-ed with the other counter words and the round key, the key advanced by
// the Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct Ctr4 {
    uint32_t a, b, c, d;
};

__host__ __device__ __forceinline__ Ctr4 philox4x32_10(Ctr4 x, uint32_t key_lo, uint32_t key_hi)
{
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    constexpr uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
#ifdef __CUDA_ARCH__
        const uint32_t hiA = __umulhi(kMulA, x.a), hiB = __umulhi(kMulB, x.c);
#else
        const uint32_t hiA = (uint32_t)(((uint64_t)kMulA * x.a) >> 32);
        const uint32_t hiB = (uint32_t)(((uint64_t)kMulB * x.c) >> 32);
#endif
        const uint32_t loA = kMulA * x.a, loB = kMulB * x.c;
        x = Ctr4{hiB ^ x.b ^ key_lo, loB, hiA ^ x.d ^ key_hi, loA};
        key_lo += kWeylA;
        key_hi += kWeylB;
    }
    return x;
}

// Stream tags (fourth counter word).
enum : uint32_t { kTagOStep = 0u, kTagInitVel = 1u, kTagSeeding = 2u, kTagMlp = 3u };

// Uniform in (0, 1): (b + 1/2) 2^-32.
__device__ __forceinline__ float unit_open_f(uint32_t b)
{
    return fmaf((float)b, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
}
__device__ __forceinline__ double unit_open_d(uint32_t b)
{
    return ((double)b + 0.5) * 2.3283064365386963e-10;
}

// Box-Muller on the two pairs of one block: (u0, u1) -> n0 = rho cos, n1 = rho sin.
template <typename R> struct Normal4 {
    R n0, n1, n2, n3;
};

// FP32 form with the hardware approximations: ln u via __logf, and
// cos/sin(2 pi u) = -cos/-sin(2 pi (u - 1/2)) via __sincosf on [-pi, pi),
// where its absolute error is about 2^-21.
__device__ __forceinline__ Normal4<float> box_muller(Ctr4 b, float)
{
    const float r0 = sqrtf(-2.0f * __logf(unit_open_f(b.a)));
    const float r1 = sqrtf(-2.0f * __logf(unit_open_f(b.c)));
    float s0, c0, s1, c1;
    __sincosf(6.28318530717958648f * (unit_open_f(b.b) - 0.5f), &s0, &c0);
    __sincosf(6.28318530717958648f * (unit_open_f(b.d) - 0.5f), &s1, &c1);
    return {-r0 * c0, -r0 * s0, -r1 * c1, -r1 * s1};
}
__device__ __forceinline__ Normal4<double> box_muller(Ctr4 b, double)
{
    const double r0 = sqrt(-2.0 * log(unit_open_d(b.a)));
    const double r1 = sqrt(-2.0 * log(unit_open_d(b.c)));
    double s0, c0, s1, c1;
    sincospi(2.0 * unit_open_d(b.b), &s0, &c0);
    sincospi(2.0 * unit_open_d(b.d), &s1, &c1);
    return {r0 * c0, r0 * s0, r1 * c1, r1 * s1};
}

template <typename R>
__device__ __forceinline__ Normal4<R> philox_normals(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                                                     uint32_t c3)
{
    return box_muller(philox4x32_10(Ctr4{c0, c1, c2, c3}, (uint32_t)seed, (uint32_t)(seed >> 32)), R(0));
}

// Device error flags (bit set in a global int).
enum : int { kErrNonFinite = 1, kErrBadArgs = 2, kErrTimeout = 4 };

}  // namespace pmf
