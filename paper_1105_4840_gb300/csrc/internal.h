// Internal host-side interfaces of libpmf (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace pmf {

// Host copy of one chain (FP64, as given by the caller).
struct ChainHost {
    int N = 0;
    std::vector<double> sigma, epsilon, charge, mass, dih_k, dih_phase, pos0;
    double bond_k = 0, bond_r0 = 0, angle_k = 0, angle_theta0 = 0, coulomb_k = 0;
    int nonbonded = 1;
};

// Tiling of N beads into 32-bead tiles; the last tile has width 8, 16 or 32.
struct ChainGeometry {
    int N = 0, Np = 0, n_tiles = 0, w_last = 32;
};

// One ring unit of the nonbonded phase: i-tile I against j-tile J, ring
// steps [tb, te); flags bit 0 = diagonal tile, bit 1 = neighbouring tiles
// (exclusions |i - j| <= 2 possible).
struct UnitDesc {
    int I, J, tb, te, flags;
};

constexpr int kChainUnitPiece = 8;  // ring steps per scheduled unit
ChainGeometry chain_geometry(int N);
std::vector<std::vector<UnitDesc>> chain_schedule(int N, int NW, int piece);

// Everything one launch of a simulation kernel needs about the run.
struct RunLaunch {
    void *state = nullptr;         // per-replica state (layout owned by the model)
    float *xout = nullptr;         // x samples
    const double *lambda = nullptr;
    const long long *nsteps_w = nullptr, *nequil_w = nullptr, *off_w = nullptr, *tw = nullptr;
    int *err = nullptr;
    double *force_out = nullptr;
    long long step_begin = 0, step_end = 0;
    int replicas = 0, stride = 1, n_blocks = 0;
    uint32_t uid_base = 0;
    unsigned long long seed = 0;
    double k = 0, kT = 1, dt = 0, gamma = 1;
};

class ChainModel {
public:
    struct Impl;
    ChainModel();
    ~ChainModel();
    cudaError_t init(const ChainHost &h, int precision);
    cudaError_t launch(const RunLaunch &L, cudaStream_t st);
    int n_beads() const;
    int n_padded() const;
    int precision() const;
    size_t state_bytes_per_replica() const;
    size_t smem_bytes() const;

private:
    Impl *p;
};

struct Od1dParams {
    double a = 2.0, x0 = -1.0;
};
cudaError_t od1d_launch(const Od1dParams &m, const RunLaunch &L, int n_rep, cudaStream_t st);

// FP64 reductions of x samples into the estimators.
struct ReduceLayout {
    const float *x = nullptr;          // device samples
    const double *lambda = nullptr;    // device [s]
    const long long *off_w = nullptr;  // device [s]
    const long long *tw = nullptr;     // device [s]
    int n_windows = 0, replicas = 0;
    double k = 0, kT = 1;
};
// Device output block: 14 arrays of n_windows doubles, in this order.
enum ResultField {
    kResLambda = 0, kResJE, kResFluct, kResG, kResCom, kResUnc, kResSeJE, kResSeFluct,
    kResVarZW, kResWMean, kResAccForce, kResMeanX, kResVarX, kResGamma2, kResFields
};
// scratch: device buffer of reduce_scratch_bytes(); out: device [kResFields][n_windows]
size_t reduce_scratch_bytes(int n_windows, int replicas);
cudaError_t reduce_launch(const ReduceLayout &L, void *scratch, double *out, cudaStream_t st);
// Allocation-free reduction: scratch in a fixed device array, equal samples
// per window, all pointers on the device.
constexpr int kNoAllocMaxWindows = 1024;
constexpr long long kNoAllocMaxWindowReplicas = 65536;  // n_windows * replicas
cudaError_t reduce_noalloc_launch(const float *x, const double *lambda, int n_windows, int replicas,
                                  long long samples_per_window, double k, double kT, double *out, cudaStream_t st);
cudaError_t work_samples_launch(const ReduceLayout &L, int mode, long long samples_per_replica, double *out,
                                cudaStream_t st);

cudaError_t philox_launch(unsigned long long seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int n,
                          uint32_t *raw, float *normals, cudaStream_t st);

}  // namespace pmf
