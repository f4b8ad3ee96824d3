// Restrained Langevin sampling of a bead chain, one CTA per replica.
//
// Parallel pulling protocol (Sec. III (ii)): every (window lambda_i, replica)
// pair is an independent simulation of H(lambda_i, x) = H_o + k/2 (x - lambda_i)^2
// (Eq. (3)) started from the same state x_o; the reaction coordinate x (here
// the end-to-end distance |r_{N-1} - r_0|) is recorded every `stride` steps
// after `n_equil` steps (Sec. IV A: every 0.1 ps).
//
// Design (sm_103a):
//  * the replica's positions, pair parameters, velocities and force buffers
//    live in shared memory for the whole launch; the step loop runs inside
//    the kernel (persistent over steps), two CTA barriers per step;
//  * nonbonded all-pairs forces use Newton's third law on 32-bead tiles: a
//    warp holds 32 i-beads in registers and walks a ring over the j-tile,
//    lane l pairing with j = (l + t) mod W at step t; the j-force accumulator
//    travels one lane per step with a warp shuffle, so every pair is
//    evaluated once and no atomics are needed.  A ragged last tile uses a
//    ring of width 8 or 16.  j data come from a duplicated tile copy in shared
//    memory so the ring index needs no wrap;
//  * each warp accumulates into its own force buffer; the bead owner sums the
//    buffers (deterministic order), so a run is bit-reproducible;
//  * bonded terms (bond, angle, three-term dihedral) are computed once by the
//    thread owning their first bead, written to per-owner slots and gathered;
//  * BAOAB with Philox4x32-10 noise, counter (bead, uid, step, 0).
#include <algorithm>
#include <memory>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace pmf {

template <typename R> struct alignas(4 * sizeof(R)) Vec4 {
    R x, y, z, w;
};
template <typename R> struct alignas(2 * sizeof(R)) Vec2 {
    R x, y;
};

template <typename R> struct ChainArgs {
    const Vec4<R> *bead_pos0;  // [Np] start state, w = sigma/2; pads far away
    const Vec2<R> *bead_eq;    // [Np] (sqrt(24 eps), q sqrt(ke)); zero for pads
    const R *bead_invm;        // [Np] 1/m, 0 for pads
    const Vec4<R> *dih;        // [N] (K1 cos d1, K2 cos d2, K3 cos d3, nonzero)
    Vec4<R> *state;            // [n_rep][2][Np] positions, velocities
    float *xout;               // samples
    const double *lambda;      // [n_windows]
    const long long *nsteps_w; // [n_windows]
    const long long *nequil_w; // [n_windows]
    const long long *off_w;    // [n_windows] first sample of the window
    const long long *tw;       // [n_windows] samples per replica
    const int4 *units;         // [NW][max_units]
    const int *unit_count;     // [NW]
    int *err;
    double *force_out;         // optional [N][3]: forces at the final positions
    const double *start;       // optional [n_rep][N][3]: start positions instead of x_o
    unsigned long long *queue; // persistent mode: next work item (zeroed before the launch)
    int *done;                 // persistent mode: [n_rep] segments finished (zeroed)
    long long n_items;         // persistent mode: n_rep x segments
    long long queue_start;     // persistent mode: first item taken (0; > 0 only to test the bounded wait)
    unsigned long long wait_ns;  // persistent mode: longest wait for a replica's previous segment
    const volatile int *abort;   // host-mapped flag: non-zero asks every CTA to stop at its next item
    int n_rep, seg_steps, persistent;
    double *wout;              // constant-velocity pulling: accumulated work at the records
    int smd;                   // constant-velocity pulling: the trap advances smd_vdt per step
    double smd_vdt;            //   after the window's equilibration
    int sequential;            // sequential protocol: every simulation visits the windows in order,
    long long window_steps;    //   window_steps steps each, in subs_per_window segments of
    int subs_per_window;       //   at most seg_steps steps
    long long step_begin, step_end;
    int N, Np, n_tiles, w_last, replicas, max_units, stride;
    uint32_t uid_base;
    unsigned long long seed;
    R k, kT, dt, gamma;
    R kb, r0, kth, th0;
    int has_angles, has_dih, nonbonded;
    int static_in_smem;        // copy the schedule and the dihedral constants into shared memory
};

template <typename R> __device__ __forceinline__ R rsqrt_r(R v);
template <> __device__ __forceinline__ float rsqrt_r<float>(float v) { return rsqrtf(v); }
template <> __device__ __forceinline__ double rsqrt_r<double>(double v) { return rsqrt(v); }

template <typename R> struct V3 {
    R x, y, z;
};
template <typename R> __device__ __forceinline__ V3<R> sub(V3<R> a, V3<R> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename R> __device__ __forceinline__ V3<R> add(V3<R> a, V3<R> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename R> __device__ __forceinline__ V3<R> scl(V3<R> a, R s) { return {a.x * s, a.y * s, a.z * s}; }
template <typename R> __device__ __forceinline__ R dot(V3<R> a, V3<R> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename R> __device__ __forceinline__ V3<R> cross(V3<R> a, V3<R> b)
{
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// FP32 uses the packed f32x2 pair engine; FP64 the scalar ring pieces.
template <typename R> constexpr bool kPacked = false;
template <> constexpr bool kPacked<float> = true;

// Shared-memory views of one replica.
template <typename R> struct Smem {
    Vec4<R> *posd;   // [n_tiles][64]: tile copy then its duplicate
    Vec2<R> *eqd;    // [n_tiles][64]
    Vec4<R> *vel;    // [Np]
    Vec4<R> *fw;     // [NW][Np]
    Vec4<R> *bslot;  // [4][Np]
    R *noise;        // [2][4 * n_blocks] normals of an O-step (by step parity), dof d = 3 b + axis
    Vec2<R> *mass;   // [Np] (1/m, c2 sqrt(kT/m)) of the O-step, per run
    const Vec4<R> *dih;  // [N] dihedral constants
    const int4 *units;   // [NW][max_units] the nonbonded schedule
    const int *ucount;   // [NW]
    // (shared-memory copies made once per CTA when the chain leaves room for
    // them, else the arguments' global arrays)
    // FP32 packed path: entry p of tile T pairs ring positions p and p + D
    // (D = pair_offset(W)): posa[64T + p] = (x_p, x_{p+D}, y_p, y_{p+D}),
    // posb[64T + p] = (z_p, z_{p+D}, s_p, s_{p+D}),
    // eqp[64T + p] = (e_p, e_{p+D}, q_p, q_{p+D}), p < 2W.  Each is a
    // contiguous float4 array, so a warp reading consecutive entries takes the
    // minimum four shared-memory wavefronts.
    float4 *posa;
    float4 *posb;
    float4 *eqp;
    int *flag;
};

// Offset between the two ring steps a packed FP32 double step evaluates.
__host__ __device__ constexpr int pair_offset(int W) { return W == 32 ? 8 : W / 2; }

__device__ __forceinline__ int tile_width(int t, int n_tiles, int w_last) { return t == n_tiles - 1 ? w_last : 32; }

template <typename R> __device__ __forceinline__ V3<R> pos_of(const Smem<R> &s, int b)
{
    const Vec4<R> p = s.posd[(b >> 5) * 64 + (b & 31)];
    return {p.x, p.y, p.z};
}

template <typename R>
__device__ __forceinline__ void store_pos(const Smem<R> &s, int b, V3<R> p, R sig, int n_tiles, int w_last)
{
    const int t = b >> 5, i = b & 31, W = tile_width(t, n_tiles, w_last);
    const Vec4<R> v{p.x, p.y, p.z, sig};
    s.posd[t * 64 + i] = v;
    s.posd[t * 64 + i + W] = v;
}

// The packed copy of one tile, rebuilt by the warp that owns the tile after
// its positions moved: lane e < W writes entries e and e + W from its own
// bead (ring position e) and the bead at ring position e + D, fetched with a
// shuffle; every lane of the warp takes part (lanes >= W only supply data).
__device__ __forceinline__ void pack_tile(const Smem<float> &s, int t, int lane, int W, V3<float> p, float sig)
{
    const int D = pair_offset(W);
    const int src = (lane + D) & (W - 1);
    const float qx = __shfl_sync(0xffffffffu, p.x, src);
    const float qy = __shfl_sync(0xffffffffu, p.y, src);
    const float qz = __shfl_sync(0xffffffffu, p.z, src);
    const float qs = __shfl_sync(0xffffffffu, sig, src);
    if (lane < W) {
        float4 *pa = s.posa + 64 * t, *pb = s.posb + 64 * t;
        const float4 lo = make_float4(p.x, qx, p.y, qy), hi = make_float4(p.z, qz, sig, qs);
        pa[lane] = lo;
        pb[lane] = hi;
        pa[lane + W] = lo;
        pb[lane + W] = hi;
    }
}

// Ring pieces.  A piece runs ring steps t = TB .. TB+NST-1 of a j-tile of
// width W against one i-tile (or two, DUAL, sharing the j loads and the
// j-force shuffles).  Lane l holds i = I*32 + l and pairs with
// j = J*32 + ((l mod W) + t) mod W; the j-force accumulator moves to lane
// l-1 (mod W) after every step.  Masks exist only where they can bite: the
// exclusions |i - j| <= 2 at t < 3 of neighbouring tiles, and the half step
// t = W/2 of a diagonal tile (which would count each pair twice).
struct PieceKind {
    int W, TB, NST, DIAG;
};
__host__ __device__ constexpr PieceKind piece_kind(int k)
{
    return k == 0 ? PieceKind{32, 0, 8, 0} : k == 1 ? PieceKind{32, 8, 8, 0} : k == 2 ? PieceKind{32, 16, 8, 0}
         : k == 3 ? PieceKind{32, 24, 8, 0} : k == 4 ? PieceKind{32, 1, 8, 1} : k == 5 ? PieceKind{32, 9, 8, 1}
         : k == 6 ? PieceKind{16, 0, 8, 0} : k == 7 ? PieceKind{16, 8, 8, 0} : k == 8 ? PieceKind{16, 1, 8, 1}
         : k == 9 ? PieceKind{8, 0, 8, 0} : PieceKind{8, 1, 4, 1};
}

template <typename R>
__device__ __forceinline__ R pair_fr(const Vec4<R> &pi, const Vec2<R> &qi, const Vec4<R> &pj, const Vec2<R> &qj, R &dx,
                                     R &dy, R &dz)
{
    dx = pj.x - pi.x;
    dy = pj.y - pi.y;
    dz = pj.z - pi.z;
    const R r2 = dx * dx + dy * dy + dz * dz;
    const R ri = rsqrt_r(r2);
    const R ri2 = ri * ri;
    const R sg = pi.w + pj.w;
    const R x2 = sg * sg * ri2;
    const R x6 = x2 * x2 * x2;
    const R lj = (qi.x * qj.x) * x6 * (R(2) * x6 - R(1));  // 24 eps_ij (2 x^12 - x^6)
    return ((qi.y * qj.y) * ri + lj) * ri2;                 // -dU/dr / r
}

template <typename R, int KIND, bool DUAL>
__device__ __forceinline__ void ring_piece(const Smem<R> &s, Vec4<R> *fw, int I1, int I2, int J, bool near1,
                                           bool near2, int wI, int lane)
{
    constexpr PieceKind K = piece_kind(KIND);
    constexpr int W = K.W, TB = K.TB, NST = K.NST;
    constexpr bool DIAG = K.DIAG;
    const int lr = lane & (W - 1);
    const bool ion = lane < wI;
    Vec4<R> pi1{R(-1e4), R(-1e4), R(-1e4), R(0)}, pi2{R(-2e4), R(-1e4), R(-1e4), R(0)};
    Vec2<R> qi1{R(0), R(0)}, qi2{R(0), R(0)};
    if (ion) {
        pi1 = s.posd[I1 * 64 + lane];
        qi1 = s.eqd[I1 * 64 + lane];
    }
    if (DUAL) {
        pi2 = s.posd[I2 * 64 + lane];
        qi2 = s.eqd[I2 * 64 + lane];
    }
    R f1x = 0, f1y = 0, f1z = 0, f2x = 0, f2y = 0, f2z = 0, fjx = 0, fjy = 0, fjz = 0;
    const Vec4<R> *pj = s.posd + J * 64 + lr;
    const Vec2<R> *qj = s.eqd + J * 64 + lr;
    const int src = (lane & ~(W - 1)) | ((lr + 1) & (W - 1));
#pragma unroll
    for (int k = 0; k < NST; ++k) {
        const int t = TB + k;
        const Vec4<R> pjv = pj[t];
        const Vec2<R> qjv = qj[t];
        R dx, dy, dz;
        R fr = pair_fr(pi1, qi1, pjv, qjv, dx, dy, dz);
        if (t < 3 && near1) {
            const int d = I1 * 32 + lane - (J * 32 + ((lr + t) & (W - 1)));
            if (d <= 2 && d >= -2) fr = R(0);
        }
        if (DIAG && 2 * t == W && lr >= (W >> 1)) fr = R(0);
        f1x -= fr * dx; f1y -= fr * dy; f1z -= fr * dz;
        fjx += fr * dx; fjy += fr * dy; fjz += fr * dz;
        if (DUAL) {
            R ex, ey, ez;
            R gr = pair_fr(pi2, qi2, pjv, qjv, ex, ey, ez);
            if (t < 3 && near2) {
                const int d = I2 * 32 + lane - (J * 32 + ((lr + t) & (W - 1)));
                if (d <= 2 && d >= -2) gr = R(0);
            }
            f2x -= gr * ex; f2y -= gr * ey; f2z -= gr * ez;
            fjx += gr * ex; fjy += gr * ey; fjz += gr * ez;
        }
        if (k + 1 < NST) {
            fjx = __shfl_sync(0xffffffffu, fjx, src);
            fjy = __shfl_sync(0xffffffffu, fjy, src);
            fjz = __shfl_sync(0xffffffffu, fjz, src);
        }
    }
    if (ion) {
        Vec4<R> f = fw[I1 * 32 + lane];
        f.x += f1x; f.y += f1y; f.z += f1z;
        fw[I1 * 32 + lane] = f;
    }
    if (DUAL) {
        Vec4<R> f = fw[I2 * 32 + lane];
        f.x += f2x; f.y += f2y; f.z += f2z;
        fw[I2 * 32 + lane] = f;
    }
#pragma unroll
    for (int o = W; o < 32; o <<= 1) {
        fjx += __shfl_xor_sync(0xffffffffu, fjx, o);
        fjy += __shfl_xor_sync(0xffffffffu, fjy, o);
        fjz += __shfl_xor_sync(0xffffffffu, fjz, o);
    }
    if (lane < W) {
        const int bj = J * 32 + ((lr + TB + NST - 1) & (W - 1));
        Vec4<R> f = fw[bj];
        f.x += fjx; f.y += fjy; f.z += fjz;
        fw[bj] = f;
    }
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Quad pieces (FP32): lane l holds two neighbouring i-beads of its ring,
// i1 at ring index l and i2 at l + 1, and at ring step t meets the j-beads at
// ring positions l + t (stream a) and l + t + D (stream b).  i1 sees ring
// offsets t and t + D, i2 sees t - 1 and t + D - 1, so odd steps t cover all
// offsets of an off-diagonal j-ring (even steps 2..W/2 the half ring of a
// diagonal tile).  Four pairs per lane and step share one set of j loads and
// one rotation (by two lanes) of the j-force streams, halving the shared
// loads and shuffles per pair; the two i-beads form the packed f32x2 operand.
//
// SPLIT pieces jump from ring step TB + 6 to TB + 16 halfway (offsets 0..15
// then 16..31 of an off-diagonal W 32 ring in one piece): the j-force streams
// then rotate by ten lanes once instead of two.
template <int W, int NST, bool SPLIT>
__device__ __forceinline__ void quad_piece(const Smem<float> &s, Vec4<float> *fw, int I, int J, int TB, bool diag,
                                           bool near, int wI, int lane)
{
    constexpr int D = pair_offset(W);
    const int lr = lane & (W - 1);
    const int l2 = (lane & ~(W - 1)) | ((lr + 1) & (W - 1));  // lane of i2 within the i-tile
    const bool on1 = lane < wI, on2 = l2 < wI;
    Vec4<float> p1{-1e4f, -1e4f, -1e4f, 0.f}, p2{-2e4f, -1e4f, -1e4f, 0.f};
    Vec2<float> q1{0.f, 0.f}, q2{0.f, 0.f};
    if (on1) { p1 = s.posd[I * 64 + lane]; q1 = s.eqd[I * 64 + lane]; }
    if (on2) { p2 = s.posd[I * 64 + l2]; q2 = s.eqd[I * 64 + l2]; }
    // i-bead data duplicated across the packed halves (streams a, b)
    const float2 nx1 = f2(-p1.x, -p1.x), ny1 = f2(-p1.y, -p1.y), nz1 = f2(-p1.z, -p1.z);
    const float2 nx2 = f2(-p2.x, -p2.x), ny2 = f2(-p2.y, -p2.y), nz2 = f2(-p2.z, -p2.z);
    const float2 s1 = f2(p1.w, p1.w), s2 = f2(p2.w, p2.w);
    const float2 e1 = f2(q1.x, q1.x), e2 = f2(q2.x, q2.x), c1 = f2(q1.y, q1.y), c2 = f2(q2.y, q2.y);
    const float2 two = f2(2.f, 2.f), mone = f2(-1.f, -1.f);
    float2 f1x = f2(0.f, 0.f), f1y = f1x, f1z = f1x, f2x = f1x, f2y = f1x, f2z = f1x;
    float2 fjx = f1x, fjy = f1x, fjz = f1x;
    const float4 *PA = s.posa + 64 * J + lr, *PB = s.posb + 64 * J + lr;
    const float4 *E = s.eqp + 64 * J + lr;
    const int src = (lane & ~(W - 1)) | ((lr + 2) & (W - 1));
    const int src_jump = (lane & ~(W - 1)) | ((lr + 10) & (W - 1));
    const int gi1 = I * 32 + lane, gi2 = I * 32 + l2;
    const bool mask_near = near && TB < 4;
    const bool mask_half = diag && lr >= (W >> 1);
#pragma unroll
    for (int k = 0; k < NST; ++k) {
        const int t = TB + 2 * k + ((SPLIT && 2 * k >= NST) ? 8 : 0);
        const float4 a = PA[t], b = PB[t], e = E[t];
        const float2 xj = f2(a.x, a.y), yj = f2(a.z, a.w), zj = f2(b.x, b.y), sj = f2(b.z, b.w);
        const float2 ej = f2(e.x, e.y), cj = f2(e.z, e.w);
        // pairs of i1 with (j_a, j_b)
        const float2 dx1 = __fadd2_rn(xj, nx1), dy1 = __fadd2_rn(yj, ny1), dz1 = __fadd2_rn(zj, nz1);
        // pairs of i2 with (j_a, j_b)
        const float2 dx2 = __fadd2_rn(xj, nx2), dy2 = __fadd2_rn(yj, ny2), dz2 = __fadd2_rn(zj, nz2);
        float2 r21 = __fmul2_rn(dx1, dx1), r22 = __fmul2_rn(dx2, dx2);
        r21 = __ffma2_rn(dy1, dy1, r21); r22 = __ffma2_rn(dy2, dy2, r22);
        r21 = __ffma2_rn(dz1, dz1, r21); r22 = __ffma2_rn(dz2, dz2, r22);
        const float2 ri1 = f2(rsqrtf(r21.x), rsqrtf(r21.y)), ri2_ = f2(rsqrtf(r22.x), rsqrtf(r22.y));
        const float2 iq1 = __fmul2_rn(ri1, ri1), iq2 = __fmul2_rn(ri2_, ri2_);
        const float2 sg1 = __fadd2_rn(s1, sj), sg2 = __fadd2_rn(s2, sj);
        const float2 x21 = __fmul2_rn(__fmul2_rn(sg1, sg1), iq1), x22 = __fmul2_rn(__fmul2_rn(sg2, sg2), iq2);
        const float2 x61 = __fmul2_rn(__fmul2_rn(x21, x21), x21), x62 = __fmul2_rn(__fmul2_rn(x22, x22), x22);
        const float2 lj1 = __fmul2_rn(__fmul2_rn(__fmul2_rn(e1, ej), x61), __ffma2_rn(x61, two, mone));
        const float2 lj2 = __fmul2_rn(__fmul2_rn(__fmul2_rn(e2, ej), x62), __ffma2_rn(x62, two, mone));
        float2 fr1 = __fmul2_rn(__ffma2_rn(__fmul2_rn(c1, cj), ri1, lj1), iq1);
        float2 fr2 = __fmul2_rn(__ffma2_rn(__fmul2_rn(c2, cj), ri2_, lj2), iq2);
        if (mask_near && t < 4) {  // exclusions |i - j| <= 2 can only meet stream a at ring offsets <= 2
            const int gj = J * 32 + ((lr + t) & (W - 1));
            const int d1 = gi1 - gj, d2 = gi2 - gj;
            if (d1 <= 2 && d1 >= -2) fr1.x = 0.f;
            if (d2 <= 2 && d2 >= -2) fr2.x = 0.f;
        }
        if (mask_half && k == NST - 1) fr1.y = 0.f;  // offset W/2 of a diagonal: counted from one side only
        f1x = __ffma2_rn(fr1, dx1, f1x); f1y = __ffma2_rn(fr1, dy1, f1y); f1z = __ffma2_rn(fr1, dz1, f1z);
        f2x = __ffma2_rn(fr2, dx2, f2x); f2y = __ffma2_rn(fr2, dy2, f2y); f2z = __ffma2_rn(fr2, dz2, f2z);
        fjx = __ffma2_rn(fr1, dx1, fjx); fjy = __ffma2_rn(fr1, dy1, fjy); fjz = __ffma2_rn(fr1, dz1, fjz);
        fjx = __ffma2_rn(fr2, dx2, fjx); fjy = __ffma2_rn(fr2, dy2, fjy); fjz = __ffma2_rn(fr2, dz2, fjz);
        if (k + 1 < NST) {
            const int sl = (SPLIT && 2 * (k + 1) == NST) ? src_jump : src;
            fjx.x = __shfl_sync(0xffffffffu, fjx.x, sl);
            fjx.y = __shfl_sync(0xffffffffu, fjx.y, sl);
            fjy.x = __shfl_sync(0xffffffffu, fjy.x, sl);
            fjy.y = __shfl_sync(0xffffffffu, fjy.y, sl);
            fjz.x = __shfl_sync(0xffffffffu, fjz.x, sl);
            fjz.y = __shfl_sync(0xffffffffu, fjz.y, sl);
        }
    }
    if (on1) {
        Vec4<float> f = fw[I * 32 + lane];
        f.x -= f1x.x + f1x.y; f.y -= f1y.x + f1y.y; f.z -= f1z.x + f1z.y;
        fw[I * 32 + lane] = f;
    }
    if (on2) {  // l2 is a permutation of the lanes: distinct beads within this pass
        Vec4<float> f = fw[I * 32 + l2];
        f.x -= f2x.x + f2x.y; f.y -= f2y.x + f2y.y; f.z -= f2z.x + f2z.y;
        fw[I * 32 + l2] = f;
    }
#pragma unroll
    for (int o = W; o < 32; o <<= 1) {
        fjx.x += __shfl_xor_sync(0xffffffffu, fjx.x, o); fjx.y += __shfl_xor_sync(0xffffffffu, fjx.y, o);
        fjy.x += __shfl_xor_sync(0xffffffffu, fjy.x, o); fjy.y += __shfl_xor_sync(0xffffffffu, fjy.y, o);
        fjz.x += __shfl_xor_sync(0xffffffffu, fjz.x, o); fjz.y += __shfl_xor_sync(0xffffffffu, fjz.y, o);
    }
    if (lane < W) {
        const int tl = TB + 2 * (NST - 1) + (SPLIT ? 8 : 0);
        const int ba = J * 32 + ((lr + tl) & (W - 1));
        Vec4<float> f = fw[ba];
        f.x += fjx.x; f.y += fjy.x; f.z += fjz.x;
        fw[ba] = f;
        const int bb = J * 32 + ((lr + tl + D) & (W - 1));
        f = fw[bb];
        f.x += fjx.y; f.y += fjy.y; f.z += fjz.y;
        fw[bb] = f;
    }
}

// Diagonal of a ragged last tile (width 8 or 16), scalar, ring steps 1..W/2;
// rare (at most one per chain), so kept compact rather than unrolled.
__device__ __noinline__ void ragged_diag_piece(const Smem<float> &s, Vec4<float> *fw, int J, int W, int lane)
{
    const int lr = lane & (W - 1);
    const bool ion = lane < W;
    Vec4<float> pi{-1e4f, -1e4f, -1e4f, 0.f};
    Vec2<float> qi{0.f, 0.f};
    if (ion) {
        pi = s.posd[J * 64 + lane];
        qi = s.eqd[J * 64 + lane];
    }
    float fix = 0, fiy = 0, fiz = 0, fjx = 0, fjy = 0, fjz = 0;
    const int src = (lane & ~(W - 1)) | ((lr + 1) & (W - 1));
    const int te = W / 2 + 1;
    for (int t = 1; t < te; ++t) {
        const Vec4<float> pj = s.posd[J * 64 + lr + t];
        const Vec2<float> qj = s.eqd[J * 64 + lr + t];
        float dx, dy, dz;
        float fr = pair_fr(pi, qi, pj, qj, dx, dy, dz);
        // |i - j| = t without wrap (excluded for t <= 2), W - t >= W/2 >= 4 with wrap;
        // at t = W/2 the upper half of the ring repeats the lower half's pairs
        if ((t < 3 && lr + t < W) || (2 * t == W && lr >= (W >> 1))) fr = 0.f;
        fix -= fr * dx; fiy -= fr * dy; fiz -= fr * dz;
        fjx += fr * dx; fjy += fr * dy; fjz += fr * dz;
        if (t + 1 < te) {
            fjx = __shfl_sync(0xffffffffu, fjx, src);
            fjy = __shfl_sync(0xffffffffu, fjy, src);
            fjz = __shfl_sync(0xffffffffu, fjz, src);
        }
    }
    if (ion) {
        Vec4<float> f = fw[J * 32 + lane];
        f.x += fix; f.y += fiy; f.z += fiz;
        fw[J * 32 + lane] = f;
    }
    for (int o = W; o < 32; o <<= 1) {
        fjx += __shfl_xor_sync(0xffffffffu, fjx, o);
        fjy += __shfl_xor_sync(0xffffffffu, fjy, o);
        fjz += __shfl_xor_sync(0xffffffffu, fjz, o);
    }
    if (lane < W) {
        const int bj = J * 32 + ((lr + te - 1) & (W - 1));
        Vec4<float> f = fw[bj];
        f.x += fjx; f.y += fjy; f.z += fjz;
        fw[bj] = f;
    }
}

// Piece kinds of the packed FP32 path (quad pieces):
//   21: W 32, t = 1, 3, 5, 7 (+8)      22: W 32, t = 17, 19, 21, 23 (+8)
//   26: W 32, t = 1, 3, 5, 7, 17, 19, 21, 23 (+8): 21 and 22 in one piece
//   23: W 32 diagonal, t = 2, 4, 6, 8 (+8)
//   24: W 16, t = 1, 3, 5, 7 (+8)       25: W 8, t = 1, 3 (+4)
//   8, 10: diagonal of a ragged tile of width 16 / 8, scalar
__device__ __forceinline__ void run_packed_piece(const Smem<float> &s, Vec4<float> *fw, int kind, int I, int J,
                                                 bool near, int wI, int lane)
{
    switch (kind) {
    case 21: quad_piece<32, 4, false>(s, fw, I, J, 1, false, near, wI, lane); break;
    case 22: quad_piece<32, 4, false>(s, fw, I, J, 17, false, near, wI, lane); break;
    case 23: quad_piece<32, 4, false>(s, fw, I, J, 2, true, near, wI, lane); break;
    case 24: quad_piece<16, 4, false>(s, fw, I, J, 1, false, near, wI, lane); break;
    case 26: quad_piece<32, 8, true>(s, fw, I, J, 1, false, near, wI, lane); break;
    case 25: quad_piece<8, 2, false>(s, fw, I, J, 1, false, near, wI, lane); break;
    case 8: ragged_diag_piece(s, fw, J, 16, lane); break;
    case 10: ragged_diag_piece(s, fw, J, 8, lane); break;
    default: break;  // the host schedule emits only the kinds above
    }
}

template <typename R, bool DUAL>
__device__ __forceinline__ void run_piece(const Smem<R> &s, Vec4<R> *fw, int kind, int I1, int I2, int J, bool n1,
                                          bool n2, int wI, int lane)
{
    switch (kind) {
    case 0: ring_piece<R, 0, DUAL>(s, fw, I1, I2, J, n1, n2, wI, lane); break;
    case 1: ring_piece<R, 1, DUAL>(s, fw, I1, I2, J, n1, n2, wI, lane); break;
    case 2: ring_piece<R, 2, DUAL>(s, fw, I1, I2, J, n1, n2, wI, lane); break;
    case 3: ring_piece<R, 3, DUAL>(s, fw, I1, I2, J, n1, n2, wI, lane); break;
    case 6: ring_piece<R, 6, DUAL>(s, fw, I1, I2, J, n1, n2, wI, lane); break;
    case 7: ring_piece<R, 7, DUAL>(s, fw, I1, I2, J, n1, n2, wI, lane); break;
    case 9: ring_piece<R, 9, DUAL>(s, fw, I1, I2, J, n1, n2, wI, lane); break;
    default:
        if (!DUAL) {
            if (kind == 4) ring_piece<R, 4, false>(s, fw, I1, I2, J, n1, n2, wI, lane);
            else if (kind == 5) ring_piece<R, 5, false>(s, fw, I1, I2, J, n1, n2, wI, lane);
            else if (kind == 8) ring_piece<R, 8, false>(s, fw, I1, I2, J, n1, n2, wI, lane);
            else if (kind == 10) ring_piece<R, 10, false>(s, fw, I1, I2, J, n1, n2, wI, lane);
        }
        break;
    }
}

// Bonded terms owned by bead t (bond t..t+1, angle t..t+2, dihedral t..t+3)
// plus the trap on the two end beads; forces go to bslot[m][t] = force on
// bead t+m.  Returns x when t is the last bead (for sampling), else -1.
template <typename R>
__device__ __forceinline__ R bonded_owner(const ChainArgs<R> &a, const Smem<R> &s, int t, R lam)
{
    const int N = a.N;
    V3<R> f0{0, 0, 0}, f1{0, 0, 0}, f2{0, 0, 0}, f3{0, 0, 0};
    const V3<R> pa = pos_of(s, t);
    R xrc = R(-1);
    if (t + 1 < N) {
        const V3<R> pb = pos_of(s, t + 1);
        const V3<R> d = sub(pb, pa);
        const R g = a.kb - a.kb * a.r0 * rsqrt_r(dot(d, d));
        f0 = add(f0, scl(d, g));
        f1 = sub(f1, scl(d, g));
        if (a.has_angles && t + 2 < N) {
            const V3<R> pc = pos_of(s, t + 2);
            const V3<R> u = sub(pa, pb), w = sub(pc, pb);
            const R lu2 = dot(u, u), lw2 = dot(w, w);
            const R inv = rsqrt_r(lu2 * lw2);
            const R inv2 = inv * inv;
            R cs = dot(u, w) * inv;
            cs = cs > R(1) ? R(1) : (cs < R(-1) ? R(-1) : cs);
            const R th = acos(cs);
            R sn2 = R(1) - cs * cs;
            sn2 = sn2 > R(1e-12) ? sn2 : R(1e-12);
            const R pref = a.kth * (th - a.th0) * rsqrt_r(sn2);
            const V3<R> ga = sub(scl(w, inv), scl(u, cs * inv2 * lw2));  // cs / |u|^2
            const V3<R> gc = sub(scl(u, inv), scl(w, cs * inv2 * lu2));  // cs / |w|^2
            f0 = add(f0, scl(ga, pref));
            f2 = add(f2, scl(gc, pref));
            f1 = sub(f1, scl(add(ga, gc), pref));
        }
        if (a.has_dih && t + 3 < N) {
            const Vec4<R> K = s.dih[t];
            if (K.w != R(0)) {
                const V3<R> pc = pos_of(s, t + 2), pd = pos_of(s, t + 3);
                const V3<R> b1 = sub(pb, pa), b2 = sub(pc, pb), b3 = sub(pd, pc);
                const V3<R> n1 = cross(b1, b2), n2 = cross(b2, b3);
                const R nn1 = dot(n1, n1), nn2 = dot(n2, n2);
                const R inv = rsqrt_r(nn1 * nn2);
                const R inv2 = inv * inv;
                const R c = dot(n1, n2) * inv;
                // U = sum_n K_n (1 + cos d_n T_n(cos phi)); T_2 = 2c^2 - 1, T_3 = 4c^3 - 3c
                const R dudc = K.x + R(4) * K.y * c + K.z * (R(12) * c * c - R(3));
                const V3<R> g1 = sub(scl(n2, inv), scl(n1, c * inv2 * nn2));  // c / |n1|^2
                const V3<R> g2 = sub(scl(n1, inv), scl(n2, c * inv2 * nn1));  // c / |n2|^2
                const V3<R> db1 = cross(b2, g1);
                const V3<R> db2 = add(cross(g1, b1), cross(b3, g2));
                const V3<R> db3 = cross(g2, b2);
                f0 = add(f0, scl(db1, dudc));
                f1 = sub(f1, scl(sub(db1, db2), dudc));
                f2 = sub(f2, scl(sub(db2, db3), dudc));
                f3 = sub(f3, scl(db3, dudc));
            }
        }
    }
    if (t == 0 || t == N - 1) {
        const V3<R> d = sub(pos_of(s, N - 1), pos_of(s, 0));
        const R x2 = dot(d, d);
        const R rx = rsqrt_r(x2);
        const R x = x2 * rx;
        const R g = a.k * (x - lam) * rx;
        if (t == 0) f0 = add(f0, scl(d, g));
        else { f0 = scl(d, -g); xrc = x; }
    }
    s.bslot[0 * a.Np + t] = Vec4<R>{f0.x, f0.y, f0.z, R(0)};
    s.bslot[1 * a.Np + t] = Vec4<R>{f1.x, f1.y, f1.z, R(0)};
    s.bslot[2 * a.Np + t] = Vec4<R>{f2.x, f2.y, f2.z, R(0)};
    s.bslot[3 * a.Np + t] = Vec4<R>{f3.x, f3.y, f3.z, R(0)};
    return xrc;
}

// Normals of O-step `step`: block b of Philox counter (b, uid, step, 0)
// gives dofs 4b..4b+3 (dof d = 3 bead + axis), stored in the noise buffer
// of the step's parity (two buffers: the next step's normals are drawn while
// the current step's are read).  Blocks [b0, b1) are spread over n_thr
// threads, this thread being number `ti`.
template <typename R>
__device__ __forceinline__ void gen_noise(const ChainArgs<R> &a, const Smem<R> &s, uint32_t uid, long long step,
                                          int b0, int b1, int ti, int n_thr)
{
    Vec4<R> *buf = reinterpret_cast<Vec4<R> *>(s.noise) + (step & 1) * ((3 * a.N + 3) >> 2);
    for (int b = b0 + ti; b < b1; b += n_thr) {
        const Normal4<R> n = philox_normals<R>(a.seed, (uint32_t)b, uid, (uint32_t)step, kTagOStep);
        buf[b] = Vec4<R>{n.n0, n.n1, n.n2, n.n3};
    }
}

// The first `early` noise blocks of the next step are drawn during the
// position update by the warps that own no tile (one block per thread); the
// rest during the force phase by the threads at the top of the CTA, which own
// few bonded terms.
__host__ __device__ __forceinline__ int early_noise_blocks(int N, int n_tiles, int NW)
{
    const int nblk = (3 * N + 3) / 4, idle = NW > n_tiles ? NW - n_tiles : 0;
    return idle * 32 < nblk ? idle * 32 : nblk;
}

// Constant-velocity pulling: trap centre at time `done` (steps completed).
__device__ __forceinline__ double smd_lambda(double lam1, double vdt, long long done, long long nequil)
{
    return done > nequil ? lam1 + vdt * (double)(done - nequil) : lam1;
}

// The accumulated work of a pulled replica lives in the unused fourth
// components of the first two velocity records (carried through the state
// record between launches and segments): FP64 directly, FP32 as an
// unevaluated sum hi + lo of two floats (about 48 bits).
__device__ __forceinline__ double work_get(const Smem<float> &s) { return (double)s.vel[0].w + (double)s.vel[1].w; }
__device__ __forceinline__ void work_set(const Smem<float> &s, double W)
{
    const float hi = (float)W;
    s.vel[0].w = hi;
    s.vel[1].w = (float)(W - (double)hi);
}
__device__ __forceinline__ double work_get(const Smem<double> &s) { return s.vel[0].w; }
__device__ __forceinline__ void work_set(const Smem<double> &s, double W) { s.vel[0].w = W; }

// The threads that simulate one replica: a whole CTA (barrier 0) or a group
// of warps of a packed CTA (named barrier `bar`, counted over its own
// threads), with the thread's index inside the team.
struct Team {
    int tid, bar, nthreads;
    __device__ __forceinline__ void sync() const
    {
        asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthreads) : "memory");
    }
};

template <typename R, int NW, bool SMD>
__device__ __forceinline__ void force_phase(const ChainArgs<R> &a, const Smem<R> &s, R lam, long long done,
                                            long long nequil, long long sample_base, bool first, uint32_t uid,
                                            long long rec, const Team &tm)
// rec: index of the x record taken at this force evaluation (the state after
// `done` steps), or -1 (records are every `stride` steps after nequil).
{
    const int tid = tm.tid, warp = tid >> 5, lane = tid & 31;
    gen_noise<R>(a, s, uid, done, first ? 0 : early_noise_blocks(a.N, a.n_tiles, NW), (3 * a.N + 3) >> 2,
                 NW * 32 - 1 - tid, NW * 32);
    for (int t = tid; t < a.N; t += NW * 32) {
        const R x = bonded_owner(a, s, t, lam);
        if (t == a.N - 1) {
            if (!(x == x) || x > R(1e30)) *s.flag = 1;
            double W = 0.0;
            if constexpr (SMD) {
                // the trap moved from lambda(done - 1) to lambda(done) = lam at
                // this x: the work of Eq. (9)
                W = work_get(s);
                if (!first && done > nequil) {
                    const double ln = smd_lambda(a.lambda[0], a.smd_vdt, done, nequil);
                    const double lo = smd_lambda(a.lambda[0], a.smd_vdt, done - 1, nequil);
                    W += 0.5 * (double)a.k * (ln - lo) * (ln + lo - 2.0 * (double)x);
                    work_set(s, W);
                }
            }
            if (rec >= 0) {
                a.xout[sample_base + rec] = (float)x;
                if constexpr (SMD) a.wout[sample_base + rec] = W;
            }
        }
    }
    if (a.nonbonded) {
        Vec4<R> *fw_mine = s.fw + warp * a.Np;
        const int cnt = s.ucount[warp];
        const int4 *u = s.units + warp * a.max_units;
        for (int q = 0; q < cnt; ++q) {
            const int4 e = u[q];  // (I1, I2 or -1, J, kind | near1 << 8 | near2 << 9)
            const int kind = e.w & 0xff;
            const bool n1 = (e.w >> 8) & 1, n2 = (e.w >> 9) & 1;
            const int wI = tile_width(e.x, a.n_tiles, a.w_last);
            if constexpr (kPacked<R>) {
                run_packed_piece(s, fw_mine, kind, e.x, e.z, n1, wI, lane);
            } else {
                if (e.y >= 0) run_piece<R, true>(s, fw_mine, kind, e.x, e.y, e.z, n1, n2, wI, lane);
                else run_piece<R, false>(s, fw_mine, kind, e.x, 0, e.z, n1, false, wI, lane);
            }
        }
    }
}

// Loads that bypass L1: a replica's state may have been written by a CTA on
// another SM (persistent mode), after this SM cached an older copy.
template <typename R> __device__ __forceinline__ Vec4<R> load_cg(const Vec4<R> *p);
template <> __device__ __forceinline__ Vec4<float> load_cg<float>(const Vec4<float> *p)
{
    const float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
    return Vec4<float>{v.x, v.y, v.z, v.w};
}
template <> __device__ __forceinline__ Vec4<double> load_cg<double>(const Vec4<double> *p)
{
    const double2 u = __ldcg(reinterpret_cast<const double2 *>(p));
    const double2 v = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    return Vec4<double>{u.x, u.y, v.x, v.y};
}

// Steps [s0, s1) of the simulation whose state record and noise stream are
// number `rep`, in window w as its replica r; the window started at step
// `origin` (0 for the parallel protocol, w x tau for the sequential one).
// State comes from x_o / the seeded start (s0 == 0) or from the replica's
// state record, and goes back to it at the end, so a replica's trajectory
// does not depend on how its steps are cut into launches or segments.
// Returns false when the run was aborted (non-finite state).
template <typename R, int NW, bool SMD>
__device__ __forceinline__ bool simulate(const ChainArgs<R> &a, const Smem<R> &s, int rep, int w, int r,
                                         long long s0, long long s1, long long origin, const Team &tm)
{
    const uint32_t uid = a.uid_base + (uint32_t)rep;
    const int tid = tm.tid;
    const R lam = (R)a.lambda[w];
    const R hdt = R(0.5) * a.dt;
    const R c1 = exp(-a.gamma * a.dt);
    const R c2 = sqrt(R(1) - c1 * c1);
    Vec4<R> *st = a.state + (size_t)rep * 2 * a.Np;

    if (tid == 0) *s.flag = 0;
    for (int b = tid; b < a.Np; b += NW * 32) {
        Vec4<R> p, v{0, 0, 0, 0};
        if (s0 == 0) {
            p = a.bead_pos0[b];
            if (a.start != nullptr && b < a.N) {
                const double *q = a.start + ((size_t)rep * a.N + b) * 3;
                p.x = (R)q[0];
                p.y = (R)q[1];
                p.z = (R)q[2];
            }
            if (b < a.N) {
                // dofs 3b..3b+2 from blocks (3b)/4 and (3b+2)/4 of counter (block, uid, 0, 1)
                const Normal4<R> n0 = philox_normals<R>(a.seed, (uint32_t)(3 * b) >> 2, uid, 0u, kTagInitVel);
                const Normal4<R> n1 = philox_normals<R>(a.seed, (uint32_t)(3 * b + 2) >> 2, uid, 0u, kTagInitVel);
                const R q[8] = {n0.n0, n0.n1, n0.n2, n0.n3, n1.n0, n1.n1, n1.n2, n1.n3};
                const int o = (3 * b) & 3;  // dof 3b + c is q[o + c] (q[4..7] = second block)
                R xi[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) xi[c] = q[o + c];
                const R sv = sqrt(a.kT * a.bead_invm[b]);
                v = Vec4<R>{sv * xi[0], sv * xi[1], sv * xi[2], R(0)};
            }
        } else {
            p = load_cg(st + b);
            p.w = a.bead_pos0[b].w;
            v = load_cg(st + a.Np + b);
        }
        store_pos<R>(s, b, V3<R>{p.x, p.y, p.z}, p.w, a.n_tiles, a.w_last);
        s.vel[b] = v;
        const R im = a.bead_invm[b];
        s.mass[b] = Vec2<R>{im, c2 * sqrt(a.kT * im)};
        for (int q = 0; q < NW; ++q) s.fw[q * a.Np + b] = Vec4<R>{0, 0, 0, 0};
        for (int m = 0; m < 4; ++m) s.bslot[m * a.Np + b] = Vec4<R>{0, 0, 0, 0};
    }
    for (int e = tid; e < a.n_tiles * 64; e += NW * 32) {
        const int t = e >> 6, i = e & 63, W = tile_width(t, a.n_tiles, a.w_last);
        if (i < 2 * W) s.eqd[e] = a.bead_eq[t * 32 + (i & (W - 1))];
    }
    tm.sync();
    if constexpr (kPacked<R>) {
        for (int e = tid; e < a.n_tiles * 64; e += NW * 32) {
            const int t = e >> 6, i = e & 63, W = tile_width(t, a.n_tiles, a.w_last), D = pair_offset(W);
            if (i >= 2 * W) continue;
            const Vec4<R> p0 = s.posd[t * 64 + (i & (W - 1))], p1 = s.posd[t * 64 + ((i + D) & (W - 1))];
            const Vec2<R> q0 = s.eqd[t * 64 + (i & (W - 1))], q1 = s.eqd[t * 64 + ((i + D) & (W - 1))];
            s.posa[e] = make_float4(p0.x, p1.x, p0.y, p1.y);
            s.posb[e] = make_float4(p0.z, p1.z, p0.w, p1.w);
            s.eqp[e] = make_float4(q0.x, q1.x, q0.y, q1.y);
        }
        tm.sync();
    }
    const long long nequil = origin + a.nequil_w[w];  // equilibration counts from the window's first step
    const long long sample_base = a.off_w[w] + (long long)r * a.tw[w];
    force_phase<R, NW, SMD>(a, s, SMD ? (R)smd_lambda(a.lambda[0], a.smd_vdt, s0, nequil) : lam, s0, nequil,
                            sample_base, true, uid, -1, tm);
    tm.sync();
    // record q is taken after nequil + (q + 1) stride steps: the first one
    // after s0 and the step it falls on (one division per segment instead
    // of a 64-bit remainder per step)
    long long rec_q = s0 >= nequil ? (s0 - nequil) / a.stride : 0;
    long long rec_step = nequil + (rec_q + 1) * a.stride;

    const int warp = tid >> 5, lane = tid & 31;
    for (long long step = s0;; ++step) {
        // one warp per 32-bead tile (warp-uniform loop: the packed copy is
        // rebuilt with shuffles by the whole warp)
        for (int tile = warp; tile < a.n_tiles; tile += NW) {
            const int b = tile * 32 + lane;
            V3<R> pnew{R(0), R(0), R(0)};
            R sig = R(0);
            if (kPacked<R> && step < s1 && b >= a.N && lane < tile_width(tile, a.n_tiles, a.w_last)) {
                const Vec4<R> pad = s.posd[tile * 64 + lane];  // pads never move
                pnew = V3<R>{pad.x, pad.y, pad.z};
                sig = pad.w;
            }
            if (b < a.N) {
                Vec4<R> F = s.bslot[b];
                if (b >= 1) { const Vec4<R> q = s.bslot[a.Np + b - 1]; F.x += q.x; F.y += q.y; F.z += q.z; }
                if (b >= 2) { const Vec4<R> q = s.bslot[2 * a.Np + b - 2]; F.x += q.x; F.y += q.y; F.z += q.z; }
                if (b >= 3) { const Vec4<R> q = s.bslot[3 * a.Np + b - 3]; F.x += q.x; F.y += q.y; F.z += q.z; }
#pragma unroll
                for (int q = 0; q < NW; ++q) {
                    const Vec4<R> g = s.fw[q * a.Np + b];
                    F.x += g.x; F.y += g.y; F.z += g.z;
                    s.fw[q * a.Np + b] = Vec4<R>{0, 0, 0, 0};
                }
                const Vec2<R> ms = s.mass[b];
                const R im = ms.x;
                Vec4<R> v = s.vel[b];
                if (step > s0) { v.x += hdt * F.x * im; v.y += hdt * F.y * im; v.z += hdt * F.z * im; }
                if (step < s1) {
                    const Vec4<R> p4 = s.posd[(b >> 5) * 64 + (b & 31)];  // position and sigma/2
                    V3<R> p{p4.x, p4.y, p4.z};
                    v.x += hdt * F.x * im; v.y += hdt * F.y * im; v.z += hdt * F.z * im;
                    p.x += hdt * v.x; p.y += hdt * v.y; p.z += hdt * v.z;
                    const R sv = ms.y;
                    const R *xi = s.noise + (step & 1) * 4 * ((3 * a.N + 3) >> 2) + 3 * b;
                    v.x = c1 * v.x + sv * xi[0];
                    v.y = c1 * v.y + sv * xi[1];
                    v.z = c1 * v.z + sv * xi[2];
                    p.x += hdt * v.x; p.y += hdt * v.y; p.z += hdt * v.z;
                    sig = p4.w;
                    store_pos<R>(s, b, p, sig, a.n_tiles, a.w_last);
                    pnew = p;
                } else if (a.force_out != nullptr) {
                    a.force_out[3 * b + 0] = (double)F.x;
                    a.force_out[3 * b + 1] = (double)F.y;
                    a.force_out[3 * b + 2] = (double)F.z;
                }
                s.vel[b] = v;
            }
            if constexpr (kPacked<R>) {
                if (step < s1) pack_tile(s, tile, lane, tile_width(tile, a.n_tiles, a.w_last), pnew, sig);
            }
        }
        if (warp >= a.n_tiles && step + 1 < s1)
            gen_noise<R>(a, s, uid, step + 1, 0, early_noise_blocks(a.N, a.n_tiles, NW), tid - a.n_tiles * 32,
                         (NW - a.n_tiles) * 32);
        if (step >= s1) break;
        tm.sync();
        long long rec = -1;
        if (step + 1 == rec_step) {
            rec = rec_q++;
            rec_step += a.stride;
        }
        force_phase<R, NW, SMD>(a, s, SMD ? (R)smd_lambda(a.lambda[0], a.smd_vdt, step + 1, nequil) : lam,
                                step + 1, nequil, sample_base, false, uid, rec, tm);
        tm.sync();
        if (*s.flag) {
            if (tid == 0) atomicOr(a.err, kErrNonFinite);
            return false;
        }
    }
    tm.sync();
    for (int b = tid; b < a.Np; b += NW * 32) {
        const V3<R> p = pos_of(s, b);
        st[b] = Vec4<R>{p.x, p.y, p.z, R(0)};
        st[a.Np + b] = s.vel[b];
    }
    return true;
}

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// The host asked the run to stop (pmf_run_wait's wall-clock limit), or a
// CTA of this run raised an error flag.
template <typename R> __device__ __forceinline__ bool stop_requested(const ChainArgs<R> &a)
{
    return *((volatile int *)a.err) != 0 || (a.abort != nullptr && *a.abort != 0);
}

// Persistent mode, thread 0: the next work item (segment-major: item =
// segment x n_rep + replica) once the replica's previous segment is done;
// -1 when the queue is empty or the run was stopped.  The wait for the
// previous segment is bounded by a.wait_ns of %globaltimer; when it runs out
// the kernel raises kErrTimeout (reported as PMF_ETIMEOUT) and every CTA
// returns at its next item.
template <typename R>
__device__ long long next_item(const ChainArgs<R> &a)
{
    if (stop_requested(a)) return -1;
    const unsigned long long it = atomicAdd(a.queue, 1ull) + (unsigned long long)a.queue_start;
    if (it >= (unsigned long long)a.n_items) return -1;
    const int rep = (int)(it % (unsigned long long)a.n_rep);
    const int seg = (int)(it / (unsigned long long)a.n_rep);
    if (seg > 0 && ld_acquire(a.done + rep) < seg) {
        const unsigned long long t0 = global_ns();
        while (ld_acquire(a.done + rep) < seg) {
            if (stop_requested(a)) return -1;
            if (global_ns() - t0 > a.wait_ns) {
                atomicOr(a.err, kErrTimeout);
                return -1;
            }
            __nanosleep(500);
        }
    }
    return (long long)it;
}

// Shared-memory views of one replica starting at p (the layout counted by
// chain_smem_bytes); *tail receives the first byte after them.  The
// schedule and the dihedral constants are read from the arguments' global
// arrays unless the caller copies them behind.
template <typename R, int NW>
__device__ __forceinline__ Smem<R> carve_smem(unsigned char *p, const ChainArgs<R> &a, unsigned char **tail)
{
    Smem<R> s;
    s.posd = reinterpret_cast<Vec4<R> *>(p); p += sizeof(Vec4<R>) * a.n_tiles * 64;
    s.eqd = reinterpret_cast<Vec2<R> *>(p); p += sizeof(Vec2<R>) * a.n_tiles * 64;
    s.vel = reinterpret_cast<Vec4<R> *>(p); p += sizeof(Vec4<R>) * a.Np;
    s.fw = reinterpret_cast<Vec4<R> *>(p); p += sizeof(Vec4<R>) * a.Np * NW;
    s.bslot = reinterpret_cast<Vec4<R> *>(p); p += sizeof(Vec4<R>) * a.Np * 4;
    s.noise = reinterpret_cast<R *>(p); p += 2 * sizeof(Vec4<R>) * ((3 * a.N + 3) >> 2);
    s.mass = reinterpret_cast<Vec2<R> *>(p); p += sizeof(Vec2<R>) * a.Np;
    s.posa = nullptr;
    s.posb = nullptr;
    s.eqp = nullptr;
    if constexpr (kPacked<R>) {
        s.posa = reinterpret_cast<float4 *>(p); p += sizeof(float4) * 64 * a.n_tiles;
        s.posb = reinterpret_cast<float4 *>(p); p += sizeof(float4) * 64 * a.n_tiles;
        s.eqp = reinterpret_cast<float4 *>(p); p += sizeof(float4) * 64 * a.n_tiles;
    }
    s.flag = reinterpret_cast<int *>(p); p += 32;  // keeps what follows 32-byte aligned
    s.dih = a.dih;
    s.units = a.units;
    s.ucount = a.unit_count;
    *tail = p;
    return s;
}

template <typename R, int NW, bool SMD>
__global__ void __launch_bounds__(NW * 32, sizeof(R) == 4 ? (NW == 4 ? 5 : (NW == 5 ? 4 : (NW == 6 ? 3 : 2))) : 1)
    chain_kernel(const ChainArgs<R> a)
// SMD: the constant-velocity pulling variant (a separate instantiation, so
// the window runs carry none of its per-step work bookkeeping).
// FP32 with 4 warps: five CTAs per SM fit; 6 and 8 warps trade occupancy for
// registers.  Two modes:
//  * one CTA per replica (blockIdx.x), steps [step_begin, step_end);
//  * persistent: gridDim.x CTAs take (segment, replica) items of seg_steps
//    steps from a global queue, so replicas migrate between CTAs and every SM
//    stays busy until the queue drains (a replica count that is not a
//    multiple of the SM count no longer leaves SMs idle).  A replica's
//    segments run in order: the CTA that takes segment q waits (bounded)
//    until segment q - 1 has released its state.  Trajectories are
//    identical in both modes.
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    __shared__ long long s_item;
    unsigned char *tail = nullptr;
    Smem<R> s = carve_smem<R, NW>(smem_raw, a, &tail);
    if (a.static_in_smem) {
        // static per-CTA data: the nonbonded schedule and the dihedral constants
        unsigned char *p = tail;
        Vec4<R> *dih = reinterpret_cast<Vec4<R> *>(p); p += sizeof(Vec4<R>) * a.N;
        int4 *units = reinterpret_cast<int4 *>(p); p += sizeof(int4) * NW * a.max_units;
        int *ucount = reinterpret_cast<int *>(p);
        for (int e = threadIdx.x; e < NW * a.max_units; e += NW * 32) units[e] = a.units[e];
        for (int e = threadIdx.x; e < NW; e += NW * 32) ucount[e] = a.unit_count[e];
        for (int b = threadIdx.x; b < a.N; b += NW * 32) dih[b] = a.dih[b];
        s.dih = dih;
        s.units = units;
        s.ucount = ucount;
    }
    // one call site of simulate() for both modes keeps the kernel compact;
    // the item survives the segment in shared memory, not in registers
    for (long long iter = 0;; ++iter) {
        if (threadIdx.x == 0) s_item = a.persistent ? next_item(a) : (iter == 0 ? (long long)blockIdx.x : -1);
        __syncthreads();
        const long long it = s_item;
        __syncthreads();  // every thread has read s_item before it is overwritten
        if (it < 0) return;
        const int rep = (int)(it % a.n_rep);
        const long long seg = it / a.n_rep;
        int w, r;
        long long s0 = a.step_begin, s1 = a.step_end, origin = 0;
        if (a.sequential) {
            // simulation rep, segment seg: part seg % subs of window seg / subs,
            // the window covering steps [w tau, (w + 1) tau)
            w = (int)(seg / a.subs_per_window);
            r = rep;
            origin = (long long)w * a.window_steps;
            s0 = origin + (seg % a.subs_per_window) * a.seg_steps;
            s1 = s0 + a.seg_steps < origin + a.window_steps ? s0 + a.seg_steps : origin + a.window_steps;
        } else {
            // parallel protocol: simulation rep is replica rep % R of window rep / R
            w = rep / a.replicas;
            r = rep % a.replicas;
            if (a.persistent) {
                s0 += seg * a.seg_steps;
                s1 = s0 + a.seg_steps < a.step_end ? s0 + a.seg_steps : a.step_end;
            } else if (stop_requested(a)) {
                return;
            }
            const long long nsteps = a.nsteps_w[w];
            s1 = s1 < nsteps ? s1 : nsteps;
        }
        const Team tm{(int)threadIdx.x, 0, NW * 32};
        if ((s0 < s1 || a.force_out != nullptr) && !simulate<R, NW, SMD>(a, s, rep, w, r, s0, s1, origin, tm)) return;
        if (a.persistent) {
            __syncthreads();  // the replica's state record is written
            if (threadIdx.x == 0) {
                const long long done_item = s_item;
                __threadfence();
                st_release(a.done + (int)(done_item % a.n_rep), (int)(done_item / a.n_rep) + 1);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

ChainGeometry chain_geometry(int N)
{
    ChainGeometry g;
    g.N = N;
    const int full = N / 32, rem = N % 32;
    if (rem == 0) {
        g.n_tiles = full;
        g.w_last = 32;
    } else {
        g.n_tiles = full + 1;
        g.w_last = rem <= 8 ? 8 : (rem <= 16 ? 16 : 32);
    }
    g.Np = (g.n_tiles - 1) * 32 + g.w_last;
    return g;
}

// Ring pieces covering every pair i < j exactly once: for each j-tile J, the
// diagonal pieces of J and the off-diagonal pieces of every i-tile I < J; two
// off-diagonal i-tiles with the same j-tile and piece kind share one DUAL
// piece.  Pieces are spread over the NW warps longest-first onto the least
// loaded warp; the bonded owners and the noise generators load warps
// 0..ceil(N/32)-1 first.
// Cost models of the FP32 schedule's longest-first assignment, in units of
// about one warp instruction: ring step, per-piece setup and flush, bonded
// pass, noise pass.  Which model balances the warps best depends on the
// chain and the warp count (the bonded and noise passes are latency-bound),
// so pmf_chain_autotune times the distinct schedules they give.
struct SchedWeights {
    double step, piece, bonded, noise;
};
constexpr SchedWeights kSchedWeights[kSchedVariants] = {
    {75, 60, 400, 250}, {75, 60, 250, 150}, {75, 60, 550, 350}, {75, 120, 400, 250}, {75, 60, 700, 400}, {75, 60, 400, 600}};

std::vector<std::vector<UnitDesc>> chain_schedule(int N, int NW, bool packed, int variant)
{
    const ChainGeometry g = chain_geometry(N);
    const SchedWeights sw = kSchedWeights[(variant >= 0 && variant < kSchedVariants) ? variant : 0];
    struct P {
        UnitDesc u;
        double cost;
    };
    std::vector<P> all;
    for (int J = 0; packed && J < g.n_tiles; ++J) {
        // packed FP32 quad pieces: 4 steps x 4 pairs per lane for a W 32 ring half
        const int W = J == g.n_tiles - 1 ? g.w_last : 32;
        if (W == 32) all.push_back(P{UnitDesc{J, -1, J, 23, 1, 0}, 4 * sw.step + sw.piece});
        else if (W == 16) all.push_back(P{UnitDesc{J, -1, J, 8, 1, 0}, 8 * 30.0 + 20.0});
        else all.push_back(P{UnitDesc{J, -1, J, 10, 1, 0}, 4 * 30.0 + 20.0});
        for (int I = 0; I < J; ++I) {
            const int nr = J - I == 1 ? 1 : 0;
            if (W == 32) {
                all.push_back(P{UnitDesc{I, -1, J, 26, nr, 0}, 8 * sw.step + sw.piece});
            } else if (W == 16) {
                all.push_back(P{UnitDesc{I, -1, J, 24, nr, 0}, 4 * sw.step + sw.piece + 10.0});
            } else {
                all.push_back(P{UnitDesc{I, -1, J, 25, nr, 0}, 2 * sw.step + sw.piece + 20.0});
            }
        }
    }
    for (int J = 0; !packed && J < g.n_tiles; ++J) {
        const int W = J == g.n_tiles - 1 ? g.w_last : 32;
        std::vector<int> diag_kinds, off_kinds;
        if (W == 32) { diag_kinds = {4, 5}; off_kinds = {0, 1, 2, 3}; }
        else if (W == 16) { diag_kinds = {8}; off_kinds = {6, 7}; }
        else { diag_kinds = {10}; off_kinds = {9}; }
        for (int k : diag_kinds) {
            const PieceKind K = piece_kind(k);
            all.push_back(P{UnitDesc{J, -1, J, k, 1, 0}, K.NST * 30.0 + 20.0});
        }
        for (int k : off_kinds) {
            const PieceKind K = piece_kind(k);
            for (int I = 0; I < J; I += 2) {
                if (I + 1 < J) {
                    all.push_back(P{UnitDesc{I, I + 1, J, k, J - I == 1 ? 1 : 0, J - I - 1 == 1 ? 1 : 0},
                                    K.NST * 55.0 + 30.0});
                } else {
                    all.push_back(P{UnitDesc{I, -1, J, k, J - I == 1 ? 1 : 0, 0}, K.NST * 30.0 + 20.0});
                }
            }
        }
    }
    std::stable_sort(all.begin(), all.end(), [](const P &x, const P &y) { return x.cost > y.cost; });
    std::vector<std::vector<UnitDesc>> per(NW);
    std::vector<double> load(NW, 0.0);
    const int nt = NW * 32;
    for (int w = 0; w < NW; ++w) {
        // bonded owners are threads 0..N-1; the noise blocks left for the
        // force phase (after those drawn during the update) run on threads
        // nt-1 downwards
        const int nblk = (3 * N + 3) / 4 - early_noise_blocks(N, g.n_tiles, NW);
        for (int pass = 0; pass * nt < N; ++pass)
            if (w * 32 < N - pass * nt) load[w] += packed ? sw.bonded : 400.0;
        for (int pass = 0; pass * nt < nblk; ++pass) {
            const int lo = nt - (nblk - pass * nt);  // lowest thread with a block in this pass
            if ((w + 1) * 32 > lo) load[w] += packed ? sw.noise : 250.0;
        }
    }
    for (const P &p : all) {
        int best = 0;
        for (int w = 1; w < NW; ++w)
            if (load[w] < load[best]) best = w;
        per[best].push_back(p.u);
        load[best] += p.cost;
    }
    return per;
}

// Shared memory of one replica CTA; `extras`: the schedule and dihedral
// copies (taken only when the total stays within kChainSmemLimit).
constexpr size_t kChainSmemLimit = 227 * 1024 - 256;
// Shared memory of one replica CTA without the static copies.
template <typename R> size_t chain_base_smem_bytes(const ChainGeometry &g, int NW)
{
    size_t b = sizeof(Vec4<R>) * g.n_tiles * 64 + sizeof(Vec2<R>) * g.n_tiles * 64 + sizeof(Vec4<R>) * g.Np * (1 + NW + 4) +
               2 * sizeof(Vec4<R>) * ((3 * g.N + 3) / 4) + sizeof(Vec2<R>) * g.Np + 32;
    if (kPacked<R>) b += sizeof(float4) * 3 * 64 * g.n_tiles;
    return b;
}
template <typename R> size_t chain_smem_bytes(const ChainGeometry &g, int NW, int max_units, bool *extras = nullptr)
{
    const size_t b = chain_base_smem_bytes<R>(g, NW);
    const size_t x = sizeof(Vec4<R>) * g.N + sizeof(int4) * NW * max_units + sizeof(int) * NW;
    const bool fit = b + x <= kChainSmemLimit;
    if (extras) *extras = fit;
    return fit ? b + x : b;
}

// Device copy of one chain in precision R.
template <typename R> struct ChainDevice {
    Vec4<R> *pos0 = nullptr;
    Vec2<R> *eq = nullptr;
    R *invm = nullptr;
    Vec4<R> *dih = nullptr;
};

template <typename R> static cudaError_t upload_chain(const ChainHost &h, const ChainGeometry &g, ChainDevice<R> &d)
{
    std::vector<Vec4<R>> pos(g.Np), dih(g.N);
    std::vector<Vec2<R>> eq(g.Np);
    std::vector<R> invm(g.Np, R(0));
    for (int b = 0; b < g.Np; ++b) {
        if (b < g.N) {
            pos[b] = Vec4<R>{(R)h.pos0[3 * b], (R)h.pos0[3 * b + 1], (R)h.pos0[3 * b + 2], (R)(0.5 * h.sigma[b])};
            eq[b] = Vec2<R>{(R)std::sqrt(24.0 * h.epsilon[b]), (R)(h.charge[b] * std::sqrt(h.coulomb_k))};
            invm[b] = (R)(1.0 / h.mass[b]);
        } else {  // pads: distinct far positions, no interaction
            pos[b] = Vec4<R>{(R)(1.0e4 + 100.0 * b), (R)1.0e4, (R)1.0e4, R(0)};
            eq[b] = Vec2<R>{R(0), R(0)};
        }
    }
    for (int b = 0; b < g.N; ++b) {
        double K[3];
        bool any = false;
        for (int m = 0; m < 3; ++m) {
            const double kk = (b + 3 < g.N) ? h.dih_k[3 * b + m] : 0.0;
            K[m] = kk * std::cos(h.dih_phase[3 * b + m]);
            any = any || kk != 0.0;
        }
        dih[b] = Vec4<R>{(R)K[0], (R)K[1], (R)K[2], (R)(any ? 1 : 0)};
    }
    cudaError_t e;
    if ((e = cudaMalloc(&d.pos0, sizeof(Vec4<R>) * g.Np)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d.eq, sizeof(Vec2<R>) * g.Np)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d.invm, sizeof(R) * g.Np)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d.dih, sizeof(Vec4<R>) * g.N)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(d.pos0, pos.data(), sizeof(Vec4<R>) * g.Np, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(d.eq, eq.data(), sizeof(Vec2<R>) * g.Np, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(d.invm, invm.data(), sizeof(R) * g.Np, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    return cudaMemcpy(d.dih, dih.data(), sizeof(Vec4<R>) * g.N, cudaMemcpyHostToDevice);
}

template <typename R> static void free_chain(ChainDevice<R> &d)
{
    cudaFree(d.pos0);
    cudaFree(d.eq);
    cudaFree(d.invm);
    cudaFree(d.dih);
    d = ChainDevice<R>{};
}

struct ChainModel::Impl {
    ChainHost host;
    ChainGeometry geo;
    int precision = 0;
    int NW = 4;
    ChainDevice<float> df;
    ChainDevice<double> dd;
    int4 *units = nullptr;
    int *unit_count = nullptr;
    int max_units = 0;
    unsigned generation = 0;
    int variant = 0;         // cost model of the FP32 schedule (kSchedWeights)
    int grid_ctas = 0;       // persistent CTAs: 0 = auto, < 0 = one CTA per replica
    int seg_steps = 1000;    // steps per persistent work item
    // schedules of the packed batch launch, per team size (warps per replica)
    struct TeamSched {
        int4 *units = nullptr;
        int *count = nullptr;
        int max_units = 0, variant = -1;
    };
    TeamSched team[17];
};

ChainModel::ChainModel() : p(new Impl) {}
ChainModel::~ChainModel()
{
    free_chain(p->df);
    free_chain(p->dd);
    cudaFree(p->units);
    cudaFree(p->unit_count);
    for (auto &t : p->team) {
        cudaFree(t.units);
        cudaFree(t.count);
    }
    delete p;
}

cudaError_t ChainModel::init(const ChainHost &h, int precision)
{
    p->host = h;
    p->geo = chain_geometry(h.N);
    p->precision = precision;
    cudaError_t e = precision == 1 ? upload_chain<double>(h, p->geo, p->dd) : upload_chain<float>(h, p->geo, p->df);
    if (e != cudaSuccess) return e;
    return set_warps(4);
}

int ChainModel::warps() const { return p->NW; }
int ChainModel::schedule_variant() const { return p->variant; }
cudaError_t ChainModel::set_schedule_variant(int v)
{
    if (v < 0 || v >= kSchedVariants) return cudaErrorInvalidValue;
    p->variant = v;
    return set_warps(p->NW);  // rebuilds the schedule (and bumps the generation)
}

cudaError_t ChainModel::set_grid(int ctas, int seg_steps)
{
    if (seg_steps < 0) return cudaErrorInvalidValue;
    p->grid_ctas = ctas;
    p->seg_steps = seg_steps > 0 ? seg_steps : 1000;
    ++p->generation;
    return cudaSuccess;
}
int ChainModel::grid_ctas() const { return p->grid_ctas; }
int ChainModel::seg_steps() const { return p->seg_steps; }
unsigned ChainModel::generation() const { return p->generation; }

cudaError_t ChainModel::set_warps(int NW)
{
    if (NW != 4 && NW != 5 && NW != 6 && NW != 8) return cudaErrorInvalidValue;
    if (p->precision == 1 && NW != 4) return cudaErrorInvalidValue;
    p->NW = NW;
    ++p->generation;
    cudaFree(p->units);
    cudaFree(p->unit_count);
    p->units = nullptr;
    p->unit_count = nullptr;
    cudaError_t e;
    const auto sched = chain_schedule(p->host.N, p->NW, p->precision != 1, p->variant);
    int mx = 1;
    for (const auto &v : sched) mx = std::max<int>(mx, (int)v.size());
    std::vector<int4> flat((size_t)p->NW * mx, int4{0, 0, 0, 0});
    std::vector<int> cnt(p->NW);
    for (int w = 0; w < p->NW; ++w) {
        cnt[w] = (int)sched[w].size();
        for (size_t q = 0; q < sched[w].size(); ++q) {
            const UnitDesc &u = sched[w][q];
            flat[(size_t)w * mx + q] =
                int4{u.I1, u.I2, u.J, u.kind | (u.near1 << 8) | (u.near2 << 9)};
        }
    }
    p->max_units = mx;
    if ((e = cudaMalloc(&p->units, sizeof(int4) * flat.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc(&p->unit_count, sizeof(int) * cnt.size())) != cudaSuccess) return e;
    if ((e = cudaMemcpy(p->units, flat.data(), sizeof(int4) * flat.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    return cudaMemcpy(p->unit_count, cnt.data(), sizeof(int) * cnt.size(), cudaMemcpyHostToDevice);
}

int ChainModel::n_beads() const { return p->geo.N; }
size_t ChainModel::smem_bytes() const
{
    return p->precision == 1 ? chain_smem_bytes<double>(p->geo, p->NW, p->max_units)
                             : chain_smem_bytes<float>(p->geo, p->NW, p->max_units);
}
int ChainModel::n_padded() const { return p->geo.Np; }
int ChainModel::precision() const { return p->precision; }

size_t ChainModel::state_bytes_per_replica() const
{
    return (p->precision == 1 ? sizeof(Vec4<double>) : sizeof(Vec4<float>)) * 2 * p->geo.Np;
}

template <typename R>
static ChainArgs<R> fill_args(const ChainModel::Impl *m, const ChainDevice<R> &d, const RunLaunch &L,
                              const int4 *units, const int *unit_count, int max_units)
{
    ChainArgs<R> a{};
    a.bead_pos0 = d.pos0;
    a.bead_eq = d.eq;
    a.bead_invm = d.invm;
    a.dih = d.dih;
    a.state = reinterpret_cast<Vec4<R> *>(L.state);
    a.xout = L.xout;
    a.lambda = L.lambda;
    a.nsteps_w = L.nsteps_w;
    a.nequil_w = L.nequil_w;
    a.off_w = L.off_w;
    a.tw = L.tw;
    a.units = units;
    a.unit_count = unit_count;
    a.err = L.err;
    a.force_out = L.force_out;
    a.start = L.start;
    a.step_begin = L.step_begin;
    a.step_end = L.step_end;
    a.N = m->geo.N;
    a.Np = m->geo.Np;
    a.n_tiles = m->geo.n_tiles;
    a.w_last = m->geo.w_last;
    a.replicas = L.replicas;
    a.max_units = max_units;
    a.stride = L.stride;
    a.uid_base = L.uid_base;
    a.seed = L.seed;
    a.k = (R)L.k;
    a.kT = (R)L.kT;
    a.dt = (R)L.dt;
    a.gamma = (R)L.gamma;
    const ChainHost &h = m->host;
    a.kb = (R)h.bond_k;
    a.r0 = (R)h.bond_r0;
    a.kth = (R)h.angle_k;
    a.th0 = (R)h.angle_theta0;
    a.has_angles = h.angle_k != 0.0;
    bool any_dih = false;
    for (int b = 0; b + 3 < h.N; ++b)
        for (int q = 0; q < 3; ++q) any_dih = any_dih || h.dih_k[3 * b + q] != 0.0;
    a.has_dih = any_dih;
    a.nonbonded = h.nonbonded;
    a.queue = L.queue;
    a.done = L.done;
    a.n_rep = L.n_blocks;
    a.seg_steps = m->seg_steps;
    a.wout = L.wout;
    a.smd = L.wout != nullptr ? 1 : 0;
    a.smd_vdt = L.smd_vdt;
    a.persistent = 0;
    a.sequential = L.sequential ? 1 : 0;
    a.window_steps = L.window_steps;
    a.subs_per_window = 1;
    if (L.sequential) {
        // a window's steps in equal segments of at most seg_steps (no segment
        // crosses a window boundary)
        const long long subs = (L.window_steps + m->seg_steps - 1) / m->seg_steps;
        a.subs_per_window = (int)subs;
        a.seg_steps = (int)((L.window_steps + subs - 1) / subs);
    }
    a.n_items = 0;
    a.queue_start = L.queue_start;
    a.wait_ns = L.wait_ns > 0 ? L.wait_ns : kDefaultSegmentWaitNs;
    a.abort = L.abort;
    a.static_in_smem = 0;
    return a;
}

template <typename R, int NW>
static cudaError_t launch_typed(ChainModel::Impl *m, const ChainDevice<R> &d, const RunLaunch &L, cudaStream_t st)
{
    if (L.smd_vdt != 0.0 && L.wout == nullptr) return cudaErrorInvalidValue;  // a pulled run records its work
    ChainArgs<R> a = fill_args<R>(m, d, L, m->units, m->unit_count, m->max_units);
    bool extras = false;
    const size_t smem = chain_smem_bytes<R>(m->geo, NW, m->max_units, &extras);
    a.static_in_smem = extras ? 1 : 0;
    void (*kern)(const ChainArgs<R>) = a.smd ? chain_kernel<R, NW, true> : chain_kernel<R, NW, false>;
    // The attribute is the kernel's upper limit, shared by every chain that
    // launches it: raise it to the device's opt-in maximum rather than to this
    // chain's size, so launches captured earlier in a graph (other chains,
    // larger footprints) stay valid.  Each CTA still gets only `smem`.
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa{};
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
    const int dyn_max = optin - (int)fa.sharedSizeBytes;  // static + dynamic <= opt-in limit
    if (smem > (size_t)dyn_max) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    if (e != cudaSuccess) return e;
    int grid = L.n_blocks;
    if (L.sequential && (L.queue == nullptr || L.done == nullptr || L.window_steps < 1 || L.step_begin != 0))
        return cudaErrorInvalidValue;
    if (L.queue != nullptr && L.done != nullptr && (m->grid_ctas >= 0 || L.sequential) && L.force_out == nullptr &&
        L.step_end > L.step_begin) {
        // persistent: as many CTAs as fit at once (or as requested), never
        // more than there are replicas
        int occ = 0, sms = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NW * 32, smem)) !=
            cudaSuccess)
            return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        const long long slots = (long long)std::max(occ, 1) * sms;
        long long want = m->grid_ctas > 0 ? m->grid_ctas : 0;
        if (want == 0) {
            // auto: fill every slot when there are enough replicas; otherwise a
            // whole number of CTAs per SM (replicas in excess of it keep the
            // queue ahead of the running segments, so no CTA waits), unless
            // that number is below 3, where more CTAs per SM still pay
            const long long per_sm = L.n_blocks / sms;
            want = L.n_blocks >= slots ? slots : (per_sm >= 3 ? per_sm * sms : L.n_blocks);
        }
        grid = (int)std::min<long long>(want, L.n_blocks);
        const long long nseg = L.sequential ? (L.step_end / L.window_steps) * a.subs_per_window
                                            : (L.step_end - L.step_begin + a.seg_steps - 1) / a.seg_steps;
        a.persistent = 1;
        a.n_items = nseg * L.n_blocks;
        if ((e = cudaMemsetAsync(L.queue, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(L.done, 0, sizeof(int) * (size_t)L.n_blocks, st)) != cudaSuccess) return e;
    }
    kern<<<grid, NW * 32, smem, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Packed persistent launch of a batch of chains (FP32)
//
// One CTA of kPackWarps warps per SM for the whole batch.  A pack is up to
// kPackWarps / G replicas of one batch item (a chain and its windows), each
// simulated by its own team of G warps with its own named barrier, side by
// side in the CTA's shared memory; G and so the number of chains per CTA
// follow from the chain's length (its shared memory per replica).  Work
// items are (segment, pack), segment-major, packs costliest first; a CTA
// takes the next item from a device queue, and the item's segment waits
// (bounded) until the pack's previous segment has stored its state.  Every
// replica runs exactly the steps, noise and force schedule (of team size G)
// it would run in a one-CTA-per-replica launch of G warps, so results are
// bit-identical to the per-chain launches with that warp count.
// ---------------------------------------------------------------------------
constexpr int kPackWarps = 16;

struct PackDesc {
    int item;       // batch item
    int first_rep;  // first replica (item-local index w * replicas + r)
    int count;      // replicas in the pack (<= kPackWarps / G)
    int G;          // warps per replica
    int slot;       // shared-memory bytes of one replica team
    int pad[3];
};

template <typename R> struct PackArgs {
    const ChainArgs<R> *items;  // per batch item: its chain's and windows' arguments, schedule of team size G
    const PackDesc *packs;      // [n_packs], costliest first
    unsigned long long *queue;  // work counter (zeroed before the launch)
    int *done;                  // [n_packs] segments finished (zeroed)
    int *err;
    const volatile int *abort;
    unsigned long long wait_ns;
    long long n_items, step_begin, step_end;
    int n_packs, seg_steps;
};

template <typename R> __device__ long long next_pack_item(const PackArgs<R> &P)
{
    auto stopped = [&] { return *((volatile int *)P.err) != 0 || (P.abort != nullptr && *P.abort != 0); };
    if (stopped()) return -1;
    const unsigned long long it = atomicAdd(P.queue, 1ull);
    if (it >= (unsigned long long)P.n_items) return -1;
    const int pk = (int)(it % (unsigned long long)P.n_packs);
    const int seg = (int)(it / (unsigned long long)P.n_packs);
    if (seg > 0 && ld_acquire(P.done + pk) < seg) {
        const unsigned long long t0 = global_ns();
        while (ld_acquire(P.done + pk) < seg) {
            if (stopped()) return -1;
            if (global_ns() - t0 > P.wait_ns) {
                atomicOr(P.err, kErrTimeout);
                return -1;
            }
            __nanosleep(500);
        }
    }
    return (long long)it;
}

template <typename R, int G>
__device__ __forceinline__ bool pack_team(const ChainArgs<R> &a, unsigned char *base, int rep, long long s0,
                                          long long s1, const Team &tm)
{
    unsigned char *tail = nullptr;
    const Smem<R> s = carve_smem<R, G>(base, a, &tail);
    return simulate<R, G, false>(a, s, rep, rep / a.replicas, rep % a.replicas, s0, s1, 0, tm);
}

template <typename R>
__global__ void __launch_bounds__(kPackWarps * 32, 1) chain_pack_kernel(const PackArgs<R> P)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    __shared__ long long s_item;
    __shared__ ChainArgs<R> s_args;
    __shared__ PackDesc s_pack;
    static_assert(sizeof(ChainArgs<R>) % sizeof(int) == 0 && sizeof(PackDesc) % sizeof(int) == 0, "copied as words");
    for (;;) {
        if (threadIdx.x == 0) s_item = next_pack_item(P);
        __syncthreads();
        const long long it = s_item;
        if (it < 0) return;
        const int pk = (int)(it % P.n_packs);
        const long long seg = it / P.n_packs;
        {
            const PackDesc *dp = P.packs + pk;
            const int *src = reinterpret_cast<const int *>(P.items + dp->item);
            for (int q = threadIdx.x; q < (int)(sizeof(ChainArgs<R>) / sizeof(int)); q += blockDim.x)
                reinterpret_cast<int *>(&s_args)[q] = src[q];
            for (int q = threadIdx.x; q < (int)(sizeof(PackDesc) / sizeof(int)); q += blockDim.x)
                reinterpret_cast<int *>(&s_pack)[q] = reinterpret_cast<const int *>(dp)[q];
        }
        __syncthreads();
        const ChainArgs<R> &a = s_args;
        const int G = s_pack.G, g = (int)(threadIdx.x >> 5) / G;
        if (g < s_pack.count) {
            const int rep = s_pack.first_rep + g;
            const long long s0 = P.step_begin + seg * P.seg_steps;
            long long s1 = s0 + P.seg_steps < P.step_end ? s0 + P.seg_steps : P.step_end;
            const long long nsteps = a.nsteps_w[rep / a.replicas];
            s1 = s1 < nsteps ? s1 : nsteps;
            const Team tm{(int)threadIdx.x - g * G * 32, 1 + g, G * 32};
            unsigned char *base = smem_raw + (size_t)g * s_pack.slot;
            if (s0 < s1) {
                switch (G) {
                case 2: pack_team<R, 2>(a, base, rep, s0, s1, tm); break;
                case 4: pack_team<R, 4>(a, base, rep, s0, s1, tm); break;
                case 8: pack_team<R, 8>(a, base, rep, s0, s1, tm); break;
                default: pack_team<R, 16>(a, base, rep, s0, s1, tm); break;
                }
            }
        }
        __syncthreads();  // every team has stored its replica's state
        if (*((volatile int *)P.err) != 0) return;
        if (threadIdx.x == 0) {
            __threadfence();
            st_release(P.done + pk, (int)seg + 1);
        }
    }
}

const int kPackTeams[4] = {2, 4, 8, 16};

cudaError_t ChainModel::team_schedule(int G, const int4 **units, const int **count, int *max_units)
{
    if (G < 1 || G > 16 || p->precision == 1) return cudaErrorInvalidValue;
    Impl::TeamSched &t = p->team[G];
    if (t.units == nullptr || t.variant != p->variant) {
        cudaFree(t.units);
        cudaFree(t.count);
        t = Impl::TeamSched{};
        const auto sched = chain_schedule(p->host.N, G, true, p->variant);
        int mx = 1;
        for (const auto &v : sched) mx = std::max<int>(mx, (int)v.size());
        std::vector<int4> flat((size_t)G * mx, int4{0, 0, 0, 0});
        std::vector<int> cnt(G);
        for (int w = 0; w < G; ++w) {
            cnt[w] = (int)sched[w].size();
            for (size_t q = 0; q < sched[w].size(); ++q) {
                const UnitDesc &u = sched[w][q];
                flat[(size_t)w * mx + q] = int4{u.I1, u.I2, u.J, u.kind | (u.near1 << 8) | (u.near2 << 9)};
            }
        }
        cudaError_t e;
        if ((e = cudaMalloc(&t.units, sizeof(int4) * flat.size())) != cudaSuccess) return e;
        if ((e = cudaMalloc(&t.count, sizeof(int) * cnt.size())) != cudaSuccess) return e;
        if ((e = cudaMemcpy(t.units, flat.data(), sizeof(int4) * flat.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        if ((e = cudaMemcpy(t.count, cnt.data(), sizeof(int) * cnt.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        t.max_units = mx;
        t.variant = p->variant;
    }
    *units = t.units;
    *count = t.count;
    *max_units = t.max_units;
    return cudaSuccess;
}

size_t ChainModel::team_slot_bytes(int G) const
{
    // one replica team without the static copies (the packed kernel reads
    // those from global memory), rounded to keep the next team 32-byte aligned
    return (chain_base_smem_bytes<float>(p->geo, G) + 31) & ~(size_t)31;
}

int pack_team_choice(const ChainModel &m, int policy)
{
    // the smallest allowed team size whose kPackWarps / G replicas fit the
    // CTA's shared memory (policy 0: G >= 4, the single-chain default;
    // 1: G >= 2; 2: G >= 8); chains too long for a full CTA at any allowed
    // size take the size that keeps the most warps busy (16 if it fits)
    const int lo = policy == 1 ? 0 : (policy == 2 ? 2 : 1);
    for (int q = lo; q < 4; ++q) {
        const int G = kPackTeams[q];
        if ((kPackWarps / G) * m.team_slot_bytes(G) <= kChainSmemLimit) return G;
    }
    for (int q = 3; q >= lo; --q)
        if (m.team_slot_bytes(kPackTeams[q]) <= kChainSmemLimit) return kPackTeams[q];
    return -1;
}

struct PackPlan {
    PackArgs<float> args{};
    ChainArgs<float> *d_items = nullptr;
    PackDesc *d_packs = nullptr;
    unsigned long long *d_queue = nullptr;
    int *d_done = nullptr;
    size_t smem = 0;
    int grid = 0;
    std::vector<int> teams;  // team size per item
    ~PackPlan()
    {
        cudaFree(d_items);
        cudaFree(d_packs);
        cudaFree(d_queue);
        cudaFree(d_done);
    }
};

cudaError_t pack_plan_create(const std::vector<PackItemSpec> &items, const std::vector<int> &teams, int seg_steps,
                             PackPlan **out)
{
    *out = nullptr;
    if (items.empty() || teams.size() != items.size() || seg_steps < 1) return cudaErrorInvalidValue;
    auto plan = std::make_unique<PackPlan>();
    std::vector<ChainArgs<float>> hargs(items.size());
    struct PC {
        PackDesc d;
        double cost;
    };
    std::vector<PC> packs;
    for (size_t m = 0; m < items.size(); ++m) {
        ChainModel &cm = *items[m].model;
        const int G = teams[m];
        if (cm.precision() == 1 || G < 2 || G > 16 || (G & (G - 1))) return cudaErrorInvalidValue;
        const int4 *units = nullptr;
        const int *count = nullptr;
        int mx = 0;
        cudaError_t e = cm.team_schedule(G, &units, &count, &mx);
        if (e != cudaSuccess) return e;
        const RunLaunch &L = items[m].L;
        if (L.sequential || L.wout != nullptr || L.force_out != nullptr || L.start != nullptr)
            return cudaErrorInvalidValue;
        hargs[m] = fill_args<float>(cm.p, cm.p->df, L, units, count, mx);
        const size_t slot32 = cm.team_slot_bytes(G);
        const int per = std::max(1, std::min(kPackWarps / G, (int)(kChainSmemLimit / slot32)));
        if (slot32 > kChainSmemLimit) return cudaErrorInvalidValue;
        const int n_rep = L.n_blocks;
        const double N = cm.n_beads();
        for (int q = 0; q * per < n_rep; ++q) {
            PackDesc d{};
            d.item = (int)m;
            d.first_rep = q * per;
            d.count = std::min(per, n_rep - q * per);
            d.G = G;
            d.slot = (int)slot32;
            packs.push_back(PC{d, (N * N * 0.5 + 40.0 * N) * d.count});
            plan->smem = std::max(plan->smem, slot32 * (size_t)per);
        }
    }
    std::stable_sort(packs.begin(), packs.end(), [](const PC &x, const PC &y) { return x.cost > y.cost; });
    std::vector<PackDesc> hp(packs.size());
    for (size_t q = 0; q < packs.size(); ++q) hp[q] = packs[q].d;
    cudaError_t e;
    if ((e = cudaMalloc(&plan->d_items, sizeof(ChainArgs<float>) * hargs.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc(&plan->d_packs, sizeof(PackDesc) * hp.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc(&plan->d_queue, sizeof(unsigned long long))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&plan->d_done, sizeof(int) * hp.size())) != cudaSuccess) return e;
    if ((e = cudaMemcpy(plan->d_items, hargs.data(), sizeof(ChainArgs<float>) * hargs.size(), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return e;
    if ((e = cudaMemcpy(plan->d_packs, hp.data(), sizeof(PackDesc) * hp.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    int dev = 0, optin = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    cudaFuncAttributes fa{};
    if ((e = cudaFuncGetAttributes(&fa, chain_pack_kernel<float>)) != cudaSuccess) return e;
    const int dyn_max = optin - (int)fa.sharedSizeBytes;
    if (plan->smem > (size_t)dyn_max) return cudaErrorInvalidValue;
    if ((e = cudaFuncSetAttribute(chain_pack_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max)) !=
        cudaSuccess)
        return e;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, chain_pack_kernel<float>, kPackWarps * 32,
                                                             plan->smem)) != cudaSuccess)
        return e;
    plan->grid = (int)std::min<long long>((long long)std::max(occ, 1) * sms, (long long)hp.size());
    PackArgs<float> &A = plan->args;
    A.items = plan->d_items;
    A.packs = plan->d_packs;
    A.queue = plan->d_queue;
    A.done = plan->d_done;
    A.err = items[0].L.err;
    A.abort = items[0].L.abort;
    A.wait_ns = items[0].L.wait_ns > 0 ? items[0].L.wait_ns : kDefaultSegmentWaitNs;
    A.n_packs = (int)hp.size();
    A.seg_steps = seg_steps;
    plan->teams = teams;
    *out = plan.release();
    return cudaSuccess;
}

cudaError_t pack_plan_launch(PackPlan *plan, long long step_begin, long long step_end, cudaStream_t st)
{
    if (!plan || step_end <= step_begin) return cudaErrorInvalidValue;
    PackArgs<float> A = plan->args;
    A.step_begin = step_begin;
    A.step_end = step_end;
    A.n_items = (long long)A.n_packs * ((step_end - step_begin + A.seg_steps - 1) / A.seg_steps);
    cudaError_t e;
    if ((e = cudaMemsetAsync(plan->d_queue, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(plan->d_done, 0, sizeof(int) * (size_t)A.n_packs, st)) != cudaSuccess) return e;
    chain_pack_kernel<float><<<plan->grid, kPackWarps * 32, plan->smem, st>>>(A);
    return cudaGetLastError();
}

void pack_plan_destroy(PackPlan *plan) { delete plan; }
int pack_plan_packs(const PackPlan *plan) { return plan ? plan->args.n_packs : 0; }
int pack_plan_grid(const PackPlan *plan) { return plan ? plan->grid : 0; }
size_t pack_plan_smem(const PackPlan *plan) { return plan ? plan->smem : 0; }

cudaError_t ChainModel::launch(const RunLaunch &L, cudaStream_t st)
{
    if (p->precision == 1) return launch_typed<double, 4>(p, p->dd, L, st);
    if (p->NW == 5) return launch_typed<float, 5>(p, p->df, L, st);
    if (p->NW == 6) return launch_typed<float, 6>(p, p->df, L, st);
    if (p->NW == 8) return launch_typed<float, 8>(p, p->df, L, st);
    return launch_typed<float, 4>(p, p->df, L, st);
}

}  // namespace pmf
