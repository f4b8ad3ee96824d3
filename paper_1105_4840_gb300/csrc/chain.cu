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
    long long step_begin, step_end;
    int N, Np, n_tiles, w_last, replicas, max_units, stride;
    uint32_t uid_base;
    unsigned long long seed;
    R k, kT, dt, gamma;
    R kb, r0, kth, th0;
    int has_angles, has_dih, nonbonded;
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

// Shared-memory views of one replica.
template <typename R> struct Smem {
    Vec4<R> *posd;   // [n_tiles][64]: tile copy then its duplicate
    Vec2<R> *eqd;    // [n_tiles][64]
    Vec4<R> *vel;    // [Np]
    Vec4<R> *fw;     // [NW][Np]
    Vec4<R> *bslot;  // [4][Np]
    int *flag;
};

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

// One ring unit: i-tile I against j-tile J for ring steps [tb, te).
template <typename R>
__device__ __forceinline__ void pair_unit(const Smem<R> &s, Vec4<R> *fw_mine, int I, int J, int tb, int te, int flags,
                                          int n_tiles, int w_last, int lane)
{
    const int wI = tile_width(I, n_tiles, w_last);
    const int W = tile_width(J, n_tiles, w_last);
    const int lr = lane & (W - 1);
    const bool ion = lane < wI;
    const bool diag = flags & 1, near = flags & 2;
    Vec4<R> pi{R(-1e4), R(-1e4), R(-1e4), R(0)};
    Vec2<R> qi{R(0), R(0)};
    if (ion) {
        pi = s.posd[I * 64 + lane];
        qi = s.eqd[I * 64 + lane];
    }
    R fix = 0, fiy = 0, fiz = 0, fjx = 0, fjy = 0, fjz = 0;
    const Vec4<R> *pj_base = s.posd + J * 64 + lr;
    const Vec2<R> *qj_base = s.eqd + J * 64 + lr;
    const int src = (lane & ~(W - 1)) | ((lr + 1) & (W - 1));
    const int gi = I * 32 + lane;
    for (int t = tb; t < te; ++t) {
        const Vec4<R> pj = pj_base[t];
        const Vec2<R> qj = qj_base[t];
        const R dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
        const R r2 = dx * dx + dy * dy + dz * dz;
        const R ri = rsqrt_r(r2);
        const R ri2 = ri * ri;
        const R sg = pi.w + pj.w;
        const R x2 = sg * sg * ri2;
        const R x6 = x2 * x2 * x2;
        const R ee = qi.x * qj.x;
        const R qq = qi.y * qj.y;
        const R lj = ee * x6 * (R(2) * x6 - R(1));
        R fr = (qq * ri + lj) * ri2;  // -dU/dr / r; force on j = fr * (rj - ri)
        if (t < 3 && near) {
            const int gj = J * 32 + ((lr + t) & (W - 1));
            const int d = gi - gj;
            if (d <= 2 && d >= -2) fr = R(0);
        }
        if (diag && 2 * t == W && lr >= (W >> 1)) fr = R(0);
        fix -= fr * dx; fiy -= fr * dy; fiz -= fr * dz;
        fjx += fr * dx; fjy += fr * dy; fjz += fr * dz;
        if (t + 1 < te) {
            fjx = __shfl_sync(0xffffffffu, fjx, src);
            fjy = __shfl_sync(0xffffffffu, fjy, src);
            fjz = __shfl_sync(0xffffffffu, fjz, src);
        }
    }
    if (ion) {
        Vec4<R> f = fw_mine[I * 32 + lane];
        f.x += fix; f.y += fiy; f.z += fiz;
        fw_mine[I * 32 + lane] = f;
    }
    for (int o = W; o < 32; o <<= 1) {
        fjx += __shfl_xor_sync(0xffffffffu, fjx, o);
        fjy += __shfl_xor_sync(0xffffffffu, fjy, o);
        fjz += __shfl_xor_sync(0xffffffffu, fjz, o);
    }
    if (lane < W) {
        const int bj = J * 32 + ((lr + te - 1) & (W - 1));
        Vec4<R> f = fw_mine[bj];
        f.x += fjx; f.y += fjy; f.z += fjz;
        fw_mine[bj] = f;
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
            R cs = dot(u, w) * inv;
            cs = cs > R(1) ? R(1) : (cs < R(-1) ? R(-1) : cs);
            const R th = acos(cs);
            R sn2 = R(1) - cs * cs;
            sn2 = sn2 > R(1e-12) ? sn2 : R(1e-12);
            const R pref = a.kth * (th - a.th0) * rsqrt_r(sn2);
            const V3<R> ga = sub(scl(w, inv), scl(u, cs / lu2));
            const V3<R> gc = sub(scl(u, inv), scl(w, cs / lw2));
            f0 = add(f0, scl(ga, pref));
            f2 = add(f2, scl(gc, pref));
            f1 = sub(f1, scl(add(ga, gc), pref));
        }
        if (a.has_dih && t + 3 < N) {
            const Vec4<R> K = a.dih[t];
            if (K.w != R(0)) {
                const V3<R> pc = pos_of(s, t + 2), pd = pos_of(s, t + 3);
                const V3<R> b1 = sub(pb, pa), b2 = sub(pc, pb), b3 = sub(pd, pc);
                const V3<R> n1 = cross(b1, b2), n2 = cross(b2, b3);
                const R nn1 = dot(n1, n1), nn2 = dot(n2, n2);
                const R inv = rsqrt_r(nn1 * nn2);
                const R c = dot(n1, n2) * inv;
                // U = sum_n K_n (1 + cos d_n T_n(cos phi)); T_2 = 2c^2 - 1, T_3 = 4c^3 - 3c
                const R dudc = K.x + R(4) * K.y * c + K.z * (R(12) * c * c - R(3));
                const V3<R> g1 = sub(scl(n2, inv), scl(n1, c / nn1));
                const V3<R> g2 = sub(scl(n1, inv), scl(n2, c / nn2));
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
        const R x = sqrt(x2);
        const R g = a.k * (x - lam) / x;
        if (t == 0) f0 = add(f0, scl(d, g));
        else { f0 = scl(d, -g); xrc = x; }
    }
    s.bslot[0 * a.Np + t] = Vec4<R>{f0.x, f0.y, f0.z, R(0)};
    s.bslot[1 * a.Np + t] = Vec4<R>{f1.x, f1.y, f1.z, R(0)};
    s.bslot[2 * a.Np + t] = Vec4<R>{f2.x, f2.y, f2.z, R(0)};
    s.bslot[3 * a.Np + t] = Vec4<R>{f3.x, f3.y, f3.z, R(0)};
    return xrc;
}

template <typename R, int NW>
__device__ __forceinline__ void force_phase(const ChainArgs<R> &a, const Smem<R> &s, R lam, long long done,
                                            long long nequil, long long sample_base, bool sample)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int t = tid; t < a.N; t += NW * 32) {
        const R x = bonded_owner(a, s, t, lam);
        if (t == a.N - 1) {
            if (!(x == x) || x > R(1e30)) *s.flag = 1;
            if (sample && done > nequil && (done - nequil) % a.stride == 0)
                a.xout[sample_base + (done - nequil) / a.stride - 1] = (float)x;
        }
    }
    if (a.nonbonded) {
        Vec4<R> *fw_mine = s.fw + warp * a.Np;
        const int cnt = a.unit_count[warp];
        const int4 *u = a.units + warp * a.max_units;
        for (int q = 0; q < cnt; ++q) {
            const int4 e = u[q];
            pair_unit<R>(s, fw_mine, e.x, e.y, e.z & 0xff, (e.z >> 8) & 0xff, e.z >> 16, a.n_tiles, a.w_last, lane);
        }
    }
}

template <typename R, int NW>
__global__ void __launch_bounds__(NW * 32) chain_kernel(const ChainArgs<R> a)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    const int rep = blockIdx.x;
    const int w = rep / a.replicas, r = rep % a.replicas;
    const uint32_t uid = a.uid_base + (uint32_t)rep;
    const long long nsteps = a.nsteps_w[w];
    const long long s0 = a.step_begin;
    const long long s1 = a.step_end < nsteps ? a.step_end : nsteps;
    if (s0 >= s1 && a.force_out == nullptr) return;
    if (*((volatile int *)a.err) != 0) return;

    Smem<R> s;
    {
        unsigned char *p = smem_raw;
        s.posd = reinterpret_cast<Vec4<R> *>(p); p += sizeof(Vec4<R>) * a.n_tiles * 64;
        s.eqd = reinterpret_cast<Vec2<R> *>(p); p += sizeof(Vec2<R>) * a.n_tiles * 64;
        s.vel = reinterpret_cast<Vec4<R> *>(p); p += sizeof(Vec4<R>) * a.Np;
        s.fw = reinterpret_cast<Vec4<R> *>(p); p += sizeof(Vec4<R>) * a.Np * NW;
        s.bslot = reinterpret_cast<Vec4<R> *>(p); p += sizeof(Vec4<R>) * a.Np * 4;
        s.flag = reinterpret_cast<int *>(p);
    }
    const int tid = threadIdx.x;
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
            if (b < a.N) {
                const Normal4<R> n = philox_normals<R>(a.seed, (uint32_t)b, uid, 0u, kTagInitVel);
                const R sv = sqrt(a.kT * a.bead_invm[b]);
                v = Vec4<R>{sv * n.n0, sv * n.n1, sv * n.n2, R(0)};
            }
        } else {
            p = st[b];
            p.w = a.bead_pos0[b].w;
            v = st[a.Np + b];
        }
        store_pos<R>(s, b, V3<R>{p.x, p.y, p.z}, p.w, a.n_tiles, a.w_last);
        s.vel[b] = v;
        for (int q = 0; q < NW; ++q) s.fw[q * a.Np + b] = Vec4<R>{0, 0, 0, 0};
        for (int m = 0; m < 4; ++m) s.bslot[m * a.Np + b] = Vec4<R>{0, 0, 0, 0};
    }
    for (int e = tid; e < a.n_tiles * 64; e += NW * 32) {
        const int t = e >> 6, i = e & 63, W = tile_width(t, a.n_tiles, a.w_last);
        if (i < 2 * W) s.eqd[e] = a.bead_eq[t * 32 + (i & (W - 1))];
    }
    __syncthreads();
    const long long nequil = a.nequil_w[w];
    const long long sample_base = a.off_w[w] + (long long)r * a.tw[w];
    force_phase<R, NW>(a, s, lam, 0, nequil, sample_base, false);
    __syncthreads();

    for (long long step = s0;; ++step) {
        for (int b = tid; b < a.N; b += NW * 32) {
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
            const R im = a.bead_invm[b];
            Vec4<R> v = s.vel[b];
            if (step > s0) { v.x += hdt * F.x * im; v.y += hdt * F.y * im; v.z += hdt * F.z * im; }
            if (step < s1) {
                V3<R> p = pos_of(s, b);
                v.x += hdt * F.x * im; v.y += hdt * F.y * im; v.z += hdt * F.z * im;
                p.x += hdt * v.x; p.y += hdt * v.y; p.z += hdt * v.z;
                const Normal4<R> n = philox_normals<R>(a.seed, (uint32_t)b, uid, (uint32_t)step, kTagOStep);
                const R sv = c2 * sqrt(a.kT * im);
                v.x = c1 * v.x + sv * n.n0;
                v.y = c1 * v.y + sv * n.n1;
                v.z = c1 * v.z + sv * n.n2;
                p.x += hdt * v.x; p.y += hdt * v.y; p.z += hdt * v.z;
                store_pos<R>(s, b, p, a.bead_pos0[b].w, a.n_tiles, a.w_last);
            } else if (a.force_out != nullptr) {
                a.force_out[3 * b + 0] = (double)F.x;
                a.force_out[3 * b + 1] = (double)F.y;
                a.force_out[3 * b + 2] = (double)F.z;
            }
            s.vel[b] = v;
        }
        if (step >= s1) break;
        __syncthreads();
        force_phase<R, NW>(a, s, lam, step + 1, nequil, sample_base, true);
        __syncthreads();
        if (*s.flag) {
            if (tid == 0) atomicOr(a.err, kErrNonFinite);
            return;
        }
    }
    __syncthreads();
    for (int b = tid; b < a.Np; b += NW * 32) {
        const V3<R> p = pos_of(s, b);
        st[b] = Vec4<R>{p.x, p.y, p.z, R(0)};
        st[a.Np + b] = s.vel[b];
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

// Ring units covering every pair i < j exactly once, split into pieces of at
// most `piece` ring steps and spread over NW warps (longest first onto the
// least loaded warp).  Bonded owners occupy warps 0..ceil(N/32)-1 first.
std::vector<std::vector<UnitDesc>> chain_schedule(int N, int NW, int piece)
{
    const ChainGeometry g = chain_geometry(N);
    std::vector<UnitDesc> all;
    for (int I = 0; I < g.n_tiles; ++I)
        for (int J = I; J < g.n_tiles; ++J) {
            const int W = J == g.n_tiles - 1 ? g.w_last : 32;
            const int tb = (I == J) ? 1 : 0;
            const int te = (I == J) ? W / 2 + 1 : W;
            const int flags = (I == J ? 1 : 0) | (J - I <= 1 ? 2 : 0);
            for (int a = tb; a < te; a += piece) all.push_back(UnitDesc{I, J, a, std::min(te, a + piece), flags});
        }
    std::stable_sort(all.begin(), all.end(),
                     [](const UnitDesc &x, const UnitDesc &y) { return (x.te - x.tb) > (y.te - y.tb); });
    std::vector<std::vector<UnitDesc>> per(NW);
    std::vector<double> load(NW, 0.0);
    const int owner_warps = std::min(NW, (N + 31) / 32);
    const int per_thread_terms = (N + NW * 32 - 1) / (NW * 32);
    for (int w = 0; w < owner_warps; ++w) load[w] += 10.0 * per_thread_terms;
    for (const UnitDesc &u : all) {
        int best = 0;
        for (int w = 1; w < NW; ++w)
            if (load[w] < load[best]) best = w;
        per[best].push_back(u);
        load[best] += (u.te - u.tb) + 0.4;
    }
    return per;
}

template <typename R> size_t chain_smem_bytes(const ChainGeometry &g, int NW)
{
    return sizeof(Vec4<R>) * g.n_tiles * 64 + sizeof(Vec2<R>) * g.n_tiles * 64 + sizeof(Vec4<R>) * g.Np * (1 + NW + 4) +
           16;
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
};

ChainModel::ChainModel() : p(new Impl) {}
ChainModel::~ChainModel()
{
    free_chain(p->df);
    free_chain(p->dd);
    cudaFree(p->units);
    cudaFree(p->unit_count);
    delete p;
}

cudaError_t ChainModel::init(const ChainHost &h, int precision)
{
    p->host = h;
    p->geo = chain_geometry(h.N);
    p->precision = precision;
    p->NW = 4;
    cudaError_t e = precision == 1 ? upload_chain<double>(h, p->geo, p->dd) : upload_chain<float>(h, p->geo, p->df);
    if (e != cudaSuccess) return e;
    const auto sched = chain_schedule(h.N, p->NW, kChainUnitPiece);
    int mx = 1;
    for (const auto &v : sched) mx = std::max<int>(mx, (int)v.size());
    std::vector<int4> flat((size_t)p->NW * mx, int4{0, 0, 0, 0});
    std::vector<int> cnt(p->NW);
    for (int w = 0; w < p->NW; ++w) {
        cnt[w] = (int)sched[w].size();
        for (size_t q = 0; q < sched[w].size(); ++q) {
            const UnitDesc &u = sched[w][q];
            flat[(size_t)w * mx + q] = int4{u.I, u.J, u.tb | (u.te << 8) | (u.flags << 16), 0};
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
    return p->precision == 1 ? chain_smem_bytes<double>(p->geo, p->NW) : chain_smem_bytes<float>(p->geo, p->NW);
}
int ChainModel::n_padded() const { return p->geo.Np; }
int ChainModel::precision() const { return p->precision; }

size_t ChainModel::state_bytes_per_replica() const
{
    return (p->precision == 1 ? sizeof(Vec4<double>) : sizeof(Vec4<float>)) * 2 * p->geo.Np;
}

template <typename R, int NW>
static cudaError_t launch_typed(ChainModel::Impl *m, const ChainDevice<R> &d, const RunLaunch &L, cudaStream_t st)
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
    a.units = m->units;
    a.unit_count = m->unit_count;
    a.err = L.err;
    a.force_out = L.force_out;
    a.step_begin = L.step_begin;
    a.step_end = L.step_end;
    a.N = m->geo.N;
    a.Np = m->geo.Np;
    a.n_tiles = m->geo.n_tiles;
    a.w_last = m->geo.w_last;
    a.replicas = L.replicas;
    a.max_units = m->max_units;
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
    const size_t smem = chain_smem_bytes<R>(m->geo, NW);
    cudaError_t e = cudaFuncSetAttribute(chain_kernel<R, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    chain_kernel<R, NW><<<L.n_blocks, NW * 32, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t ChainModel::launch(const RunLaunch &L, cudaStream_t st)
{
    if (p->precision == 1) return launch_typed<double, 4>(p, p->dd, L, st);
    return launch_typed<float, 4>(p, p->df, L, st);
}

}  // namespace pmf
