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
//   wtab    T[Q][20]            for each crystal axis a_m the Voigt vector
//                               (a1^2,a2^2,a3^2,2a2a3,2a1a3,2a1a2), 18 values padded
//                               to 20 (the adjoint's basis forms)
//   atab    T[Q][8]             the first two crystal axes a_0, a_1 in the sample
//                               frame (columns of A), padded to 8 (the sweep's zone
//                               energy)
//   cubw    float[Q][12]        FP32 MPM step: the Voigt weights (x^2, y^2, z^2, yz,
//                               xz, xy) of the first two crystal axes a_0, a_1
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

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
    double sig0;             // prescribed uniaxial stress (traction control)
    int32_t wait_timeout;    // set when a sweep gave up waiting for a tile copy
    int32_t pad1;
};

// Division by an invariant 32-bit divisor d >= 1 with one high multiply
// (Granlund & Montgomery, PLDI'94, Sec. 4): l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, t = mulhi(m, n), n / d = (t + ((n - t) >> s1)) >> s2
// with s1 = min(l, 1), s2 = max(l - 1, 0).  Exact for every 32-bit n.
struct UDiv {
    uint32_t m, s1, s2;
};
inline UDiv make_udiv(uint32_t d) {
    uint32_t l = 0;
    while (l < 31 && (1u << l) < d) ++l;
    const unsigned long long m = ((((unsigned long long)1 << l) - d) << 32) / d + 1;
    return UDiv{(uint32_t)m, l < 1 ? l : 1u, l > 0 ? l - 1 : 0u};
}

// One replica of a batch (a single handle is a batch of one).  Replica r's
// blocks, nodes and stress occupy [blk_off, blk_off + nblk) of the batch
// arrays (nodes are indexed like blocks, 3 values each; the stress of a
// replica is its own [2][6][nblk][4] array at 48 * blk_off).
struct alignas(16) Replica {   // 16 B aligned: the pipelined sweep stages it with a bulk copy
    int nx, ny, nz, nbx, nby, nbz;
    int nblk;                 // 2x2x2 blocks = MPM cells = background nodes
    int cta_off, ncta;        // its CTAs in the block-parallel grids (BLOCK_THREADS each)
    int pad;
    long long blk_off;
    uint32_t key0, key1, replica, pad2;
    double lam_sd_half;       // lambda * (S11 - S12 - S44/2) / 2
    double lam;               // lambda: MC energy per GPa of elastic energy density
    DevState *st;
    UDiv divx, divy;          // division by nbx and by nby
    uint32_t pad3;
    float lam_sd_half_f, lam_f;   // FP32 copies of the two scales
};
static_assert(sizeof(Replica) % 16 == 0, "Replica must be a whole number of 16 B units");

constexpr int BLOCK_THREADS = 256;   // threads of the sweep and stress CTAs

// MPM work decomposition of one replica for the chosen patch shape: tiles of
// owned nodes per edge and the first (tile-major, plane-minor) work item.
struct MpmSched {
    int tiles_x, tiles_y;
    long long plane_off;      // entry nrep holds the total
};

template <typename T>
struct MpmArgs {
    const Replica *reps;
    const MpmSched *sched;   // nrep + 1 entries
    int nrep;
    long long total;         // work items of the whole batch
    const uint4 *spins;
    const T *u_in;
    T *u_out;
    T *v;
    const T *ctab;           // FP64 step: rotated stiffness rows
    const float *cubw;       // FP32 step: Voigt weights of two crystal axes per orientation (12 each)
    float cub[4];            // FP32 step: C12, 2 C44, C44 and C11 - C12 - 2 C44
    int nq;                  // orientations (the FP32 step stages cubw in shared memory up to MPM_STAB_MAX)
    T dt, dt_over_m, keep;   // keep = 1 - damping
    int grid;                // persistent CTAs
};

constexpr int MPM_STAB_MAX = 1024;   // orientations whose FP32 table the MPM step holds in shared memory

// The plain (unfused, incremental) FP64 step of a single replica: point stresses
// sig[6][nblk][8] (component, cell, local point a + 2b + 4c) and cell corner forces
// fcell[24][nblk] kept in global memory between its kernels.
struct PlainArgs {
    const uint4 *spins;
    const double *ctab;
    const DevState *st;      // mean strain
    const double *u;
    double *u_out;
    double *v;
    double *sig;
    double *fcell;
    double dt, dt_over_m, keep;
    int nbx, nby, nbz, nblk;
};
cudaError_t launch_plain_init(const PlainArgs &a, cudaStream_t s);
cudaError_t launch_plain_step(const PlainArgs &a, cudaStream_t s);

template <typename T>
struct StressArgs {
    const Replica *reps;
    const int *cta_rep;      // replica of every CTA
    const uint4 *spins;
    const T *u;
    const T *ctab;
    T *sig;
    double *partials;        // 7 doubles per CTA: sum sigma (6), sum 1/2 sigma.eps
    int nctas;
};

template <typename T>
struct SweepArgs {
    const Replica *reps;
    const int *cta_rep;
    uint4 *spins;
    const T *sig;
    const T *atab;                   // the first two crystal axes per orientation (8 values)
    const unsigned long long *thr;   // integer Metropolis thresholds for dE = 0..7
    int trial, nq;
    T J, kT;
    int nctas;
    uint4 *work;                     // zone mode: trial list {site, replica, q_new | q_old << 16, r1}
    unsigned *count;                 // zone mode: entries in the list
    const T *ctab, *stab;            // constant-strain mode: stiffness and compliance rows (Q x 24)
    const T *u;                      // recompute mode: nodal displacement (the stress of a trial site
                                     // is formed from it as the stress pass would)
    int skip_copy;                   // fault injection: the stored-stress copy is never started, so its
                                     // bounded wait runs out (HMC_FAULT=sweep_wait)
    int nrep;                        // replicas; with one, the kernels read rep0 below
    int cta;                         // threads per CTA: 256, or 128 (a tile split over two CTAs; the
                                     // stored-stress point-zone and pure Potts forms)
    double *margin;                  // margin form: (H - t) / max(1, |t|) of every trial evaluated with
                                     // the elastic term, natural site order (others untouched)
    Replica rep0;                    // replica 0's descriptor, passed by value
    uint32_t rkey[20];               // with one replica: its Philox round keys (philox_round_keys)
};

// The ten round keys of Philox4x32-10 for key (k0, k1): round r uses (k0 + r W0, k1 + r W1)
// mod 2^32 with the Weyl increments W0 = 0x9E3779B9, W1 = 0xBB67AE85.
inline void philox_round_keys(uint32_t k0, uint32_t k1, uint32_t (&rk)[20]) {
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
        rk[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
}

// Elastic term of a sweep: none, one-point zone from the stored stress (constant
// traction or constant strain), or the 27-point zone (trials listed by the
// sweep, decided by the zone kernel).
enum SweepMode { SWEEP_POTTS = 0, SWEEP_POINT = 1, SWEEP_ZONE_LIST = 2, SWEEP_STRAIN = 3 };

template <typename T>
struct ZoneArgs {
    const Replica *reps;
    const uint4 *snap;               // spins at the start of the half step
    uint4 *spins;                    // live spins: accepted trials are XOR-ed in
    const T *u;                      // nodal displacement
    const T *ctab;                   // Q x 24 rotated stiffness
    const T *ktab;                   // Q x 8 x 300 element stiffness of a point per position in its cell
    const uint4 *work;
    const unsigned *count;
    const unsigned long long *thr;
    const uint16_t *sched;           // elimination schedule (zone_schedule)
    const uint16_t *scatter;         // element-matrix places per reflection and zone cell (zone_scatter_table)
    int nsched;
    T J, kT;
};

// MPM patch shapes (cells per patch edge; owned nodes = cells - 1).  A variant
// index v in [0, 2 * MPM_NSHAPES) selects shape v % MPM_NSHAPES; v >= MPM_NSHAPES
// selects the paired-FMA Hooke product (FP32 only); v = MPM_TWO_CELL is the
// 16x16 shape with two cells per thread in paired FP32 registers (FP32 only).
enum MpmShape { MPM_16x16 = 0, MPM_32x8 = 1, MPM_8x32 = 2, MPM_NSHAPES = 3, MPM_TWO_CELL = 6 };
inline int mpm_nvariants(bool fp32) { return fp32 ? MPM_TWO_CELL + 1 : MPM_NSHAPES; }
int mpm_shape_cx(int shape);
int mpm_shape_cy(int shape);

// Launchers (return cudaGetLastError of the launch).
template <typename T>
cudaError_t launch_mpm_step(const MpmArgs<T> &a, int shape, cudaStream_t s);
template <typename T>
cudaError_t launch_stress(const StressArgs<T> &a, bool store, cudaStream_t s);   // store = 0: reductions only
template <typename T>
cudaError_t launch_sweep(const SweepArgs<T> &a, int colour, int mode, bool recompute, cudaStream_t s);
// the stored-stress point-zone sweep of a single replica that also writes every evaluated
// trial's distance to its Metropolis threshold to a.margin (mode SWEEP_POINT or SWEEP_STRAIN)
template <typename T>
cudaError_t launch_sweep_margin(const SweepArgs<T> &a, int colour, int mode, cudaStream_t s);
template <typename T>
cudaError_t launch_zone(const ZoneArgs<T> &a, int grid, cudaStream_t s);
template <typename T>
int zone_per_sm();                 // resident zone CTAs per SM
cudaError_t zone_prepare();        // opt the zone kernels into their dynamic shared memory
std::vector<uint16_t> zone_schedule();   // empty if it does not fit the kernel's table
std::vector<uint16_t> zone_scatter_table(const std::vector<uint16_t> &schedule);
void zone_element_tables(const double *Cv, int Q, std::vector<double> &out);
cudaError_t mpm_prepare();  // opt the MPM kernels into their dynamic shared memory (once, before any capture)
cudaError_t sweep_prepare();  // opt the elastic sweeps into their shared memory
template <typename T>
int mpm_per_sm(int variant, int nq);  // resident MPM CTAs per SM

// One CTA per replica: fixed-order FP64 sum of its stress partials, loading
// update (update_strain) and MCS counter (advance).
// End-of-step reduction: END_GROUPS CTAs per replica sum the stress partials in a fixed
// order in FP64; the last to finish sums their group sums in group order and finishes the
// step.  Its scratch lies behind the nctas x 7 stress partials: END_GROUPS x 7 group sums
// per replica, then one arrival counter per replica (zero between launches).
constexpr int END_GROUPS = 32;
inline size_t end_scratch_doubles(int nrep) { return (size_t)nrep * END_GROUPS * 7 + (size_t)(nrep + 1) / 2; }
cudaError_t launch_end_mcs(const Replica *reps, int nrep, double *partials, int nctas, int update_strain, int advance,
                           cudaStream_t s);
cudaError_t launch_check_spins(const uint16_t *nat, long long n, int nq, DevState *st, cudaStream_t s);
cudaError_t launch_pack_spins(const uint16_t *nat, uint4 *blk, int nx, int ny, int nz, cudaStream_t s);
cudaError_t launch_unpack_spins(const uint4 *blk, uint16_t *nat, int nx, int ny, int nz, cudaStream_t s);
cudaError_t launch_bonds_counts(const uint4 *blk, int nbx, int nby, int nbz, int nq,
                                unsigned long long *counts, DevState *st, cudaStream_t s);
cudaError_t launch_grain_count(const uint4 *spins, int nbx, int nby, int nbz, unsigned *parent,
                               unsigned long long *count, int *err, cudaStream_t s);
cudaError_t launch_bins(const unsigned long long *counts, const int32_t *binmap, int nq, int nbins,
                        unsigned long long *bins, double *fractions, long long n_sites, cudaStream_t s);

}  // namespace hmc
