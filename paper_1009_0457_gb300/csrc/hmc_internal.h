// Internal declarations shared by the CUDA translation units of libhmc.
// Device-side layouts (all owned by the handle):
//   spins   uint4[nblk]         one 2x2x2 voxel block = one MPM cell; eight uint16
//                               in slot order: red (x+y+z even) local corners
//                               (000,110,101,011), then black (100,010,001,111)
//   u[2],v  T[nnodes*3]         node I = i + nbx*(j + nby*k) at voxel corner (2i,2j,2k);
//                               u ping-pongs between the two buffers each MPM step
//   sig     T[2][6][nblk][4]    stress of each colour's four points per block,
//                               component-major so that one colour and one
//                               component of a block is one 16 B (FP32) load
//   ctab    T[Q][24]            rotated stiffness C'(q), 21 upper-triangle Voigt
//                               entries (row-major) padded to 24
//   wtab    T[Q][20]            zone-energy weights: for each crystal axis a_m the
//                               Voigt vector (a1^2,a2^2,a3^2,2a2a3,2a1a3,2a1a2),
//                               18 values padded to 20
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hmc {

// Scalars that kernels read or update on the device, so that a Monte Carlo
// step needs no host round trip and can be replayed from a CUDA graph.
struct DevState {
    double ebar[6];          // mean strain (Voigt, engineering shear)
    float ebar_f[6];         // its FP32 copy for FP32 kernels
    float pad0[2];
    double mean_sigma[6];    // mean stress of the last stress pass (FP64 reduction)
    double energy;           // elastic energy of the last stress pass (FP64 reduction)
    double sr[36];           // Reuss compliance of the initial spin field
    double axN[6];           // n(x)n, Voigt tensor components
    double axNs[6];          // weights with n.sigma.n = axNs . sigma
    double axB[6];           // S_R axN
    double axNB;             // axN . axB
    double eps0;             // uniaxial strain
    int32_t bc;              // HMC_BC_*
    uint32_t mcs;            // Monte Carlo steps completed
    unsigned long long accepted;   // spin changes since the last reset
    unsigned long long unlike;     // unlike-bond count of the last statistics pass
    int32_t nonfinite;       // set when a reduction produced a non-finite value
    int32_t bad_spin;        // set by the upload check when a spin is >= Q
};

template <typename T>
struct MpmArgs {
    const uint4 *spins;
    const T *u_in;
    T *u_out;
    T *v;
    const T *ctab;
    const DevState *st;
    int nbx, nby, nbz;
    int tiles_x, tiles_y;    // 15-node tiles per edge
    int grid;                // persistent CTAs
    T dt, dt_over_m, keep;   // keep = 1 - damping
};

template <typename T>
struct StressArgs {
    const uint4 *spins;
    const T *u;
    const T *ctab;
    const DevState *st;
    T *sig;
    double *partials;        // 7 doubles per CTA: sum sigma (6), sum 1/2 sigma.eps
    int nbx, nby, nbz;
    long long nblk;
};

template <typename T>
struct SweepArgs {
    uint4 *spins;
    const T *sig;
    const T *wtab;
    const unsigned long long *thr;   // integer Metropolis thresholds for dE = 0..7
    DevState *st;
    int nx, ny, nz, nbx, nby, nbz;
    long long nblk;
    uint32_t key0, key1, replica;
    int trial, nq;
    T J, kT, lam_sd_half;            // lambda * (S11 - S12 - S44/2) / 2
};

// Launchers (return cudaGetLastError of the launch).
template <typename T>
cudaError_t launch_mpm_step(const MpmArgs<T> &a, cudaStream_t s);
template <typename T>
cudaError_t launch_stress(const StressArgs<T> &a, int grid, cudaStream_t s);
template <typename T>
cudaError_t launch_sweep(const SweepArgs<T> &a, int colour, bool elastic, cudaStream_t s);
int stress_grid(long long nblk);
cudaError_t mpm_prepare();  // opt the MPM kernel into its dynamic shared memory (once, before any capture)
int mpm_tiles(int nb);      // node tiles along one edge
template <typename T>
int mpm_grid(int nbx, int nby, int nbz, int num_sms);

cudaError_t launch_end_mcs(DevState *st, const double *partials, int nparts, long long n_sites,
                           int update_strain, int advance, cudaStream_t s);
cudaError_t launch_check_spins(const uint16_t *nat, long long n, int nq, DevState *st, cudaStream_t s);
cudaError_t launch_pack_spins(const uint16_t *nat, uint4 *blk, int nx, int ny, int nz, cudaStream_t s);
cudaError_t launch_unpack_spins(const uint4 *blk, uint16_t *nat, int nx, int ny, int nz, cudaStream_t s);
cudaError_t launch_bonds_counts(const uint4 *blk, int nbx, int nby, int nbz, int nq,
                                unsigned long long *counts, DevState *st, cudaStream_t s);
cudaError_t launch_bins(const unsigned long long *counts, const int32_t *binmap, int nq, int nbins,
                        unsigned long long *bins, double *fractions, long long n_sites, cudaStream_t s);

}  // namespace hmc
