/*
 * hmc.h -- C ABI of the GB300 (sm_103a) hybrid Monte Carlo library.
 *
 * Method: Zhang, Bartel & Lusk, "Parallelized Hybrid Monte Carlo Simulation of
 * Stress-Induced Texture Evolution".  A Q-state Potts model of grain
 * orientations on a periodic nx x ny x nz voxel lattice (Sec. "Hybrid Monte
 * Carlo Methodology", Eq. 4) evolves by red/black checkerboard Metropolis
 * sweeps (Sec. "Microstructural Evolution"; Eq. 5).  Each trial's energy change
 * is the bond-energy change plus the elastic shift of a one-point
 * constant-traction zone (Eqs. 6-8), scaled to MC units by Eq. 13.  The stress
 * comes from a time-explicit material point method (MPM) run towards the
 * quasi-static state before every Monte Carlo step (Sec. "Elastic
 * Deformation"; the loading schedule of Sec. "Results": equilibrate, then one
 * Monte Carlo step).
 *
 * Conventions shared by every entry point:
 *  - Host arrays passed in are caller-owned, read during the call and not
 *    retained.  Host arrays passed out are caller-allocated with the stated
 *    sizes.  The handle owns all device memory it uses.
 *  - Site arrays are in natural order, x fastest: p = x + nx*(y + ny*z).
 *    Node arrays (the MPM background mesh, one node per 2x2x2 voxel cell) are
 *    in natural order of nodes: I = i + (nx/2)*(j + (ny/2)*k), 3 values per
 *    node (x,y,z).  Tensors are Voigt (11,22,33,23,13,12); strains carry
 *    engineering shear, stresses tensor components.  Stress unit: GPa.
 *  - Work is ordered on the handle's stream.  Calls that return values to the
 *    host synchronise that stream before returning.
 *  - Every call returns an hmc_status; no C++ exception crosses the ABI.  A
 *    failed call leaves the handle valid; hmc_last_error() describes the
 *    failure.  CUDA errors map to HMC_ERR_CUDA, allocation failures to
 *    HMC_ERR_OOM, calls before hmc_set_orientations to HMC_ERR_STATE; a
 *    non-finite FP64 reduction (mean stress, energy) sets a per-replica flag
 *    reported as HMC_ERR_NONFINITE by the calls that read statistics or the
 *    accepted count, until hmc_set_nodal / hmc_set_state load a new state.
 *  - Host-side fault injection for tests (environment variable HMC_FAULT):
 *    "alloc" fails handle creation before any CUDA call, "launch" fails
 *    hmc_mpm_steps / hmc_mc_sweeps before anything is enqueued, "nan" writes a
 *    NaN into the first nodal displacement before the next stress pass,
 *    "sweep_wait" makes stored-stress sweeps skip their stress copy so that
 *    their bounded (1 s per CTA) wait for it runs out: HMC_ERR_TIMEOUT.
 */
#ifndef HMC_H_
#define HMC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hmc_handle hmc_handle;

typedef enum {
    HMC_OK = 0,
    HMC_ERR_ARG = -1,
    HMC_ERR_CUDA = -2,
    HMC_ERR_OOM = -3,
    HMC_ERR_STATE = -4,
    HMC_ERR_NONFINITE = -5,
    HMC_ERR_TIMEOUT = -6
} hmc_status;

/* Loading control.  UNIAXIAL: the mean strain along load_axis is held at
 * `strain` and the other five mean stresses are driven to zero once per
 * Monte Carlo step (traction-free sides of a periodic cell).  STRAIN6: all six
 * mean strain components are prescribed by `strain6`.  TRACTION: uniaxial
 * stress `stress` (GPa) along load_axis, the loading of Sec. "Results" (a cube
 * under a uniaxial tension): once per Monte Carlo step the mean strain moves by
 * the Reuss compliance of the initial volume fractions times the gap between
 * the prescribed and the mean stress; it starts at the Reuss strain of the
 * prescribed stress. */
enum { HMC_BC_UNIAXIAL = 0, HMC_BC_STRAIN6 = 1, HMC_BC_TRACTION = 2 };
/* Elastic term of the trial energy: off (pure Potts); the one-point
 * constant-traction zone shift w(q_old) - w(q_new), w(q) = 1/2 s.S'(q).s
 * (Eqs. 6-8), from the stress of the last stress pass; or the zone of the 27
 * points around the site (Eq. 6 over a zone of half-width one point, the larger
 * zone proposed in Sec. "Conclusions"): the zone is re-equilibrated with the
 * forces of the rest of the body on its nodes held at their current values, and
 * the shift is the change of its minimum potential energy,
 * 1/2 e0.dC (I + G dC)^-1 e0 with e0 the site's strain from the current nodal
 * displacement and mean strain, dC = C'(q_new) - C'(q_old), G the compliance of
 * the zone seen at the site (evaluated as the equal form 1/2 e0.dC e0 - 1/2 f.K'^+ f,
 * K' the zone stiffness with the new orientation, f = B_p^T dC e0, B_p the site's
 * strain-displacement map).  ZONE1 evaluates every trial against the spins as
 * they were at the start of the half step (the zone holds sites of the sweep's
 * own colour) and needs nx, ny, nz >= 6; it does not read the stored stress. */
enum { HMC_ELASTIC_OFF = 0, HMC_ELASTIC_TRACTION = 1, HMC_ELASTIC_ZONE1 = 2, HMC_ELASTIC_STRAIN = 3 };
/* HMC_ELASTIC_STRAIN: the one-point zone with the point's strain held fixed
 * instead of its stress (Eq. 8 read with the strain e = S'(q_old) s of the
 * stored stress): 1/2 e.(C'(q_new) - C'(q_old)).e.  It also favours the softer
 * orientation, with a different magnitude. */
/* Trial orientation: copy a random one of the six neighbours, or draw
 * uniformly from 0..Q-1. */
enum { HMC_TRIAL_NEIGHBOR = 0, HMC_TRIAL_UNIFORM_Q = 1 };
/* Arithmetic of the MPM step, the stress and the zone energy. */
enum { HMC_FP64 = 0, HMC_FP32 = 1 };
/* Texture measures of hmc_texture_histogram. */
enum { HMC_HIST_PER_Q = 0, HMC_HIST_ANGLE_100 = 1, HMC_HIST_YOUNG = 2 };

typedef struct {
    int32_t nx, ny, nz;          /* voxels per edge; even, >= 4; periodic            */
    int32_t n_orient;            /* Q, 1..65535                                       */
    double J, kT;                /* Potts bond energy and MC temperature (alpha=kT/J) */
    double c11, c12, c44;        /* cubic stiffness of the crystal frame, GPa         */
    int32_t bc;                  /* HMC_BC_*                                          */
    double load_axis[3];         /* UNIAXIAL load direction (normalised here)         */
    double strain;               /* UNIAXIAL strain along load_axis                   */
    double strain6[6];           /* STRAIN6 mean strain (Voigt, engineering shear)    */
    double elastic_scale;        /* lambda: MC energy per GPa of energy density;
                                    < 0 selects the calibration of Eqs. 11-13 with
                                    the Table 1 constants and Delta = 1/max(nx,ny,nz) */
    int32_t elastic;             /* HMC_ELASTIC_*                                     */
    int32_t trial;               /* HMC_TRIAL_*                                       */
    int32_t mpm_steps_per_mcs;   /* explicit MPM steps before each MC step, >= 0     */
    double dt;                   /* explicit time step; <= 0 selects 0.5 h / c_max   */
    double damping;              /* velocity damping per step; < 0 selects 0.05       */
    int32_t precision;           /* HMC_FP64 | HMC_FP32                               */
    uint64_t seed;               /* Philox key of the trial stream                    */
    uint32_t replica;            /* third Philox counter word (ensemble member)       */
    void *stream;                /* cudaStream_t for all work; NULL = library-owned   */
    double stress;               /* TRACTION stress along load_axis, GPa               */
    int32_t store_stress;        /* 1: the stress pass of each MC step stores every
                                    point's stress and the point-zone sweeps read it;
                                    0: the step's stress pass only forms the mean
                                    stress and energy, and the sweeps recompute the
                                    stress of each non-trivial trial site from the
                                    nodal displacement (same arithmetic, same bits).
                                    The stored field is then refreshed only by
                                    hmc_compute_stress.  2 (constant-traction point
                                    zone): the autotuner picks 1 or 0 by timing both
                                    forms at the first MPM use (the same bits either
                                    way); other elastic terms treat 2 as 1.          */
} hmc_params;

/* Scalars the library derived from the parameters, and its counters. */
typedef struct {
    double dt, damping, elastic_scale;
    double strain_bar[6];        /* current mean strain Ebar                          */
    uint32_t mcs;                /* Monte Carlo steps completed (Philox word 1)       */
    int32_t u_buffer;            /* which displacement buffer holds the current state */
    int64_t n_sites, n_nodes;
    int64_t zone_trials;         /* ZONE1: trials the last half sweep listed (all replicas) */
} hmc_info;

/* Fill *p with defaults: 32^3, Q = 64, J = 1, kT = 0.7, Ni constants
 * 246.5/147.3/124.7 GPa, uniaxial 1e-3 along z, calibrated lambda, traction
 * shift, neighbour trials, 50 MPM steps per MCS, default dt and damping,
 * FP32, seed 1, replica 0, library stream. */
void hmc_default_params(hmc_params *p);

/* Create a handle for one replica.  Validates *p (HMC_ERR_ARG on odd or small
 * edges, Q out of range, bad enums, non-finite constants, singular stiffness)
 * and allocates every device buffer for the grid.  *out is NULL on failure. */
hmc_status hmc_create(const hmc_params *p, hmc_handle **out);

/* Batched ensemble: one handle holding n_replicas independent replicas
 * (params[r] for replica r), each swept in the same launches -- every phase of
 * the Monte Carlo step (MPM step, stress, half sweeps, end of step) is one
 * launch over all replicas, replayed from one CUDA graph.  Replicas may differ
 * in nx, ny, nz, load_axis, strain, strain6, elastic_scale, seed and replica;
 * all other fields must be equal (HMC_ERR_ARG otherwise).  Each replica's
 * spins, stress and Monte Carlo stream are exactly those of the same
 * replica run alone.  hmc_create(p, out) is hmc_create_batch(p, 1, out). */
hmc_status hmc_create_batch(const hmc_params *params, int32_t n_replicas, hmc_handle **out);

/* Select the replica that the per-replica accessors act on (hmc_set_spins,
 * hmc_get_spins, hmc_get/set_stress, hmc_get/set_nodal, hmc_get/set_strain,
 * hmc_texture_histogram, hmc_energy, hmc_get_info, hmc_get/set_state);
 * replica 0 after creation. */
hmc_status hmc_select_replica(hmc_handle *h, int32_t r);

/* Launch configuration chosen by the autotuner at the first MPM step (or the
 * default before it): MPM variant v (patch shape v % 3 -- 0: 16x16 cells,
 * 1: 32x8, 2: 8x32 -- with, for v >= 3 (FP32 only), the Hooke product as
 * paired FP32 FMAs) and the number of persistent MPM CTAs.  The autotuner
 * times every candidate on scratch copies of the nodal state; all patch
 * shapes of one Hooke variant give bit-identical results.  Environment
 * variable HMC_AUTOTUNE=0 keeps variant 0; HMC_MPM_SHAPE=<v> forces one. */
hmc_status hmc_get_tuning(hmc_handle *h, int32_t *mpm_shape, int32_t *mpm_grid);

/* The sweep choices of the autotuner, made at the same time (a library service with
 * no counterpart in the paper): *sweep_cta (nullable) the threads per half-sweep CTA,
 * 256 (one CTA per 256-block tile) or 128 (the tile split over two CTAs; the
 * stored-stress point-zone and pure Potts forms); *stored (nullable) 1 if the stress
 * pass of a Monte Carlo step stores the stress for the sweeps, 0 if the sweeps
 * recompute it (store_stress = 2 lets the tuner choose).  Every choice gives the same
 * results.  HMC_SWEEP_CTA=128|256 forces the CTA size. */
hmc_status hmc_get_sweep_tuning(hmc_handle *h, int32_t *sweep_cta, int32_t *stored);

/* Release the handle and all its device memory (NULL is a no-op). */
void hmc_destroy(hmc_handle *h);

/* Orientation table and initial spin field (Sec. "Elastic Deformation",
 * Eqs. 16-18; Sec. "Results", random initial orientations).
 *   euler_zyz: Q x 3 doubles (phi, theta, psi), radians; A = Rz(phi) Ry(theta)
 *              Rz(psi) maps crystal-frame vectors to the sample frame.
 *   spins:     N = nx*ny*nz orientation indices 0..Q-1, natural order (for a
 *              batch: every replica's field in replica order, back to back).
 * Builds the rotated stiffness C'(q) (Voigt 6x6) and the zone-energy table in
 * FP64 on the host, uploads them and the spins, zeroes the nodal displacement
 * and velocity, resets the MC step counter to 0, and sets the mean strain
 * (UNIAXIAL: strain / (n.S_R.n) S_R:(n(x)n) with S_R the Reuss compliance of
 * these spins; STRAIN6: strain6).  HMC_ERR_ARG if a spin is >= Q or an angle
 * is not finite. */
hmc_status hmc_set_orientations(hmc_handle *h, const double *euler_zyz, const uint16_t *spins);

/* Replace the spin field only (N values, natural order, each < Q); tables,
 * nodal state, mean strain and counters are kept. */
hmc_status hmc_set_spins(hmc_handle *h, const uint16_t *spins);

/* Copy the spin field out (N values, natural order). */
hmc_status hmc_get_spins(hmc_handle *h, uint16_t *spins);

/* Device-pointer forms for zero-copy exchange with other device code (for
 * example a tensor's data pointer).  The pointer must be memory of the current
 * device (device or managed), 16-byte aligned, and hold N uint16 values of the
 * selected replica in natural order; it is read or written on the handle's
 * stream and not retained.  HMC_ERR_ARG (nothing launched) for NULL, a
 * misaligned pointer or one that is not device memory of this device.
 * hmc_set_spins_dev validates the values on the device (HMC_ERR_ARG if one is
 * >= Q, spins unchanged) and packs them; hmc_get_spins_dev unpacks into the
 * buffer.  Both return after the copy has completed.
 * hmc_set_orientations_dev is hmc_set_orientations with the spins of all
 * replicas (back to back) in device memory; they pass through the host once,
 * since the Reuss compliance is formed from their volume fractions there. */
hmc_status hmc_set_spins_dev(hmc_handle *h, const uint16_t *d_spins);
hmc_status hmc_get_spins_dev(hmc_handle *h, uint16_t *d_spins);
hmc_status hmc_set_orientations_dev(hmc_handle *h, const double *euler_zyz, const uint16_t *d_spins);

/* nsteps explicit MPM steps (Sec. "Elastic Deformation"): per material point
 * strain = Ebar + sym(grad u) from the trilinear nodal field, stress =
 * C'(q) strain (Eq. 1), internal nodal force -sum_p V sigma_p.gradN, then
 * v <- (1 - damping) v + dt f / m and u <- u + dt v on the periodic mesh.
 * If elastic_energy is not NULL, the stress of the final state is computed
 * (as hmc_compute_stress) and its elastic energy written there. */
hmc_status hmc_mpm_steps(hmc_handle *h, int32_t nsteps, double *elastic_energy);

/* Stress of every point from the current displacement, stored on the device
 * for the sweeps; optionally returns the mean stress (6) and the elastic
 * energy sum_p 1/2 sigma_p.eps_p (one voxel volume per point), each reduced
 * in FP64 across the domain.  Either pointer may be NULL. */
hmc_status hmc_compute_stress(hmc_handle *h, double *mean_stress, double *elastic_energy);

/* One red/black half sweep (Sec. "Microstructural Evolution"): the four sites
 * of `colour` ((x+y+z) even = 0 = red) in each 2x2x2 block share one
 * Philox4x32-10 block with counter (s, mcs, replica, 2 + colour) and key seed,
 * s the index of the block's origin site; the site with the j-th smallest local
 * corner index lx + 2 ly + 4 lz takes word w = word j.  A neighbour trial picks
 * neighbour floor(6 w / 2^32) (order -x, +x, -y, +y, -z, +z) and takes the low
 * 32 bits of 6 w as its acceptance draw; a trial over all orientations picks
 * floor(Q w / 2^32) and takes word j of a second block (counter word 3 =
 * 4 + colour).  The trial is accepted by Eq. 5 on J*(change of unlike-neighbour
 * count) plus lambda times the stored-stress zone shift.  The MC step counter is not advanced.
 * *accepted (nullable) receives the number of sites that changed.  A
 * stored-stress sweep waits for its asynchronous stress copy with a 1 s limit
 * per CTA; a CTA whose wait ran out changes no spin and, before it returns,
 * waits (bounded, 20 further limits) for the copy to land, so that no copy
 * outlives it.  The next call that reads the accepted count or the statistics
 * reports HMC_ERR_TIMEOUT once, and later sweeps run normally.  Should a copy
 * still be outstanding after those limits (valid device memory always
 * arrives, so only a failing device gets there), HMC_ERR_TIMEOUT says so and
 * every later call on the handle returns HMC_ERR_STATE: destroy it. */
hmc_status hmc_sweep_half(hmc_handle *h, int32_t colour, int64_t *accepted);

/* The same half sweep (single-replica handle, point-zone elastic term, stored
 * stress), which also reports how close each decision was: margin (N doubles,
 * HOST, natural order) receives (H - t) / max(1, |t|) for every trial that was
 * evaluated with the elastic term -- H = J dE + dH_e the energy change and
 * t = -kT ln u the threshold of Eq. 5 in the handle's precision, accepted iff
 * H <= t -- and NaN for every other site.  A diagnostic for stating the error
 * of the FP32 path: a decision that differs between precisions is one whose
 * margin is within that precision's rounding.  Allocates and frees a device
 * buffer of N doubles per call and synchronises.  HMC_ERR_ARG for a batch, a
 * NULL margin, or a handle whose sweeps do not read the stored stress. */
hmc_status hmc_sweep_half_margins(hmc_handle *h, int32_t colour, double *margin, int64_t *accepted);

/* The same explicit steps in the plain form of Sec. "Elastic Deformation", kept as
 * the baseline the fused step is measured against: nodal velocities give each
 * point's strain increment, Hooke's law (Eq. 1) updates the point's stress by it,
 * and the stresses give the internal nodal forces -- three unfused kernels per step
 * (forces per cell, node update, stress increments per cell) with every point's
 * stress (6 doubles) and every cell's corner forces (24 doubles) stored in global
 * memory between them.  Each call starts the point stresses from the total form
 * C'(q)(Ebar + B u) of the current state, so while the spins are fixed it advances
 * u and v as hmc_mpm_steps does, to FP64 rounding.  Single-replica FP64 handles
 * only (HMC_ERR_ARG otherwise); the stress and force buffers (64 doubles per cell)
 * are allocated by the first call and kept with the handle.  Stream-ordered; the
 * stored stress that the sweeps read is not changed. */
hmc_status hmc_mpm_steps_plain(hmc_handle *h, int32_t nsteps);

/* Close a Monte Carlo step: with UNIAXIAL control update the mean strain from
 * the mean stress of the last hmc_compute_stress, then advance the counter. */
hmc_status hmc_end_mcs(hmc_handle *h);

/* n_mcs Monte Carlo steps, each: mpm_steps_per_mcs MPM steps, stress, red
 * half sweep, black half sweep (stress frozen over the step), end of step.
 * This is the loading schedule of Sec. "Results" (in every load sub-step the
 * quasi-static elastic state is obtained by the explicit MPM of Sec. "Elastic
 * Deformation", then one Monte Carlo step follows) with the red/black update of
 * Sec. "Microstructural Evolution".  Replayed from a captured CUDA graph (the
 * first call on each displacement buffer captures it; make that call before any
 * capture of your own).  *accepted (nullable) receives the number of spin
 * changes over all n_mcs steps and all replicas.  HMC_ERR_STATE before
 * hmc_set_orientations; HMC_ERR_ARG for n_mcs < 0; HMC_ERR_NONFINITE or
 * HMC_ERR_TIMEOUT as described at hmc_sweep_half and hmc_compute_stress. */
hmc_status hmc_mc_sweeps(hmc_handle *h, int32_t n_mcs, int64_t *accepted);

/* Texture of the current spin field (Sec. "Results").  counts_per_q (Q int64,
 * nullable): volume of each orientation, summing exactly to N.  fractions
 * (nbins doubles, nullable) by kind: PER_Q: nbins = Q, counts / N;
 * ANGLE_100: angle between the load axis and the nearest crystal <100> in
 * bins of 90/nbins degrees; YOUNG: E(load axis)/c11 in nbins equal bins
 * between the <100> and <111> moduli.  Counts are int64, fractions FP64. */
hmc_status hmc_texture_histogram(hmc_handle *h, int32_t kind, int32_t nbins, double *fractions,
                                 int64_t *counts_per_q);

/* Grain count of the selected replica (Sec. "Microstructural Evolution": a
 * grain's volume is the number of grid sites it holds; the mean grain volume
 * of the grain-growth law V^(3/2) = c2 t is N / *n_grains).  A grain is a set of
 * sites of one orientation connected through face neighbours on the periodic
 * lattice.  Synchronous; union-find on the device in a buffer of 4 bytes per
 * site of the largest replica, allocated by the first call.  HMC_ERR_TIMEOUT if
 * a union-find loop reached its iteration cap (no result). */
hmc_status hmc_grain_count(hmc_handle *h, int64_t *n_grains);

/* Statistics of the current state.  unlike_bonds: the number of unlike
 * nearest-neighbour bonds of the periodic lattice, each bond counted once
 * (int64), so that the boundary energy of the Potts Hamiltonian (Eq. 4, read
 * as J (1 - delta) per bond) is J times it.  elastic_energy: sum over the points
 * of 1/2 sigma.eps (Eq. 1, V = one voxel) and mean_stress (6, Voigt) from the
 * last stored stress pass, both reduced in FP64 in a fixed order.  Any pointer
 * may be NULL.  HMC_ERR_NONFINITE if the reduction was not finite. */
hmc_status hmc_energy(hmc_handle *h, int64_t *unlike_bonds, double *elastic_energy, double *mean_stress);

/* Stored stress of every point (N x 6 doubles, natural order): the stress of
 * the last pass that stored it -- hmc_compute_stress always, a Monte Carlo step
 * only when its sweeps read it (point-zone elastic term and store_stress = 1).
 * hmc_set_stress replaces it (rounded to the handle's precision), so that a
 * stored-stress sweep can be run on a given stress. */
hmc_status hmc_get_stress(hmc_handle *h, double *sigma);
hmc_status hmc_set_stress(hmc_handle *h, const double *sigma);

/* Nodal displacement and velocity (nnodes x 3 doubles each; either NULL). */
hmc_status hmc_get_nodal(hmc_handle *h, double *u, double *v);
hmc_status hmc_set_nodal(hmc_handle *h, const double *u, const double *v);

/* New scalar load of the selected replica, e.g. one substep of a loading
 * ramp: the uniaxial strain (UNIAXIAL) or stress in GPa (TRACTION).  The mean
 * strain moves at once by the Reuss response to the change (UNIAXIAL: along
 * S_R n(x)n to the new axial strain; TRACTION: by S_R (change) n(x)n); the
 * control loop then acts at the end of each Monte Carlo step.  HMC_ERR_ARG for
 * STRAIN6 (use hmc_set_strain) or a non-finite value.  The load is a parameter,
 * not part of hmc_get_state. */
hmc_status hmc_set_load(hmc_handle *h, double value);

/* Mean strain Ebar (6, Voigt engineering). */
hmc_status hmc_get_strain(hmc_handle *h, double *strain_bar);
hmc_status hmc_set_strain(hmc_handle *h, const double *strain_bar);

/* Derived scalars and counters. */
hmc_status hmc_get_info(hmc_handle *h, hmc_info *info);

/* Checkpoint: spins, nodal u and v, mean strain and the MC step counter.  With
 * buf == NULL, *bytes receives the size; otherwise *bytes must be at least
 * that size.  The counter-based stream makes a resumed run bit-identical. */
hmc_status hmc_get_state(hmc_handle *h, void *buf, size_t *bytes);
hmc_status hmc_set_state(hmc_handle *h, const void *buf, size_t bytes);

/* Allocation-free stress pass (no counterpart in the paper; a library
 * service).  For callers that cannot allocate device memory where they need
 * the stress -- code inside another framework's memory pool or a fixed-budget
 * arena, or code that must not call cudaMalloc/cudaFree because those calls
 * synchronise the device.  Computes what hmc_compute_stress and
 * hmc_get_stress give (stress of every point in FP32; mean stress and elastic
 * energy reduced in FP64) from caller-owned DEVICE buffers, and allocates
 * nothing: its only scratch, the per-CTA partial sums of the fixed-order
 * reduction, lives in a static 512 KiB device array that every GPU loading
 * the library holds until the process exits.
 *   d_spins   N = nx*ny*nz orientation indices, natural order (device)
 *   d_u       (nx/2)(ny/2)(nz/2) x 3 nodal displacements, FP32 (device)
 *   d_ctab    Q x 36 rotated stiffness C'(q), full Voigt 6x6 row-major, FP32 (device)
 *   strain_bar  6 doubles (HOST), mean strain, Voigt engineering shear
 *   d_sigma   N x 6 FP32 output, natural order (device)
 *   d_mean    6 doubles output (device);  d_energy  1 double output (device)
 *   stream    cudaStream_t, NULL = legacy default stream
 * Grids of at most 16,777,216 points (2,097,152 cells; 256^3 is the largest
 * cube accepted) are served; larger ones are rejected with HMC_ERR_ARG.  Work
 * is enqueued on `stream` and not waited for.  The first call on a device
 * looks up the scratch array's device address (cudaGetSymbolAddress) with that
 * device current and keeps it for the life of the process: make that first
 * call before any stream capture, in the device's primary context, and do not
 * call cudaDeviceReset afterwards (the kept address would be stale).  All
 * calls share the one scratch array, which keeps the last call's partial sums:
 * calls whose work can overlap on the GPU (different streams with no ordering
 * between them) race, so order them.  Errors are reported through
 * hmc_last_error(NULL). */
hmc_status hmc_stress_noalloc(const uint16_t *d_spins, const float *d_u, const float *d_ctab,
                              const double *strain_bar, int32_t nx, int32_t ny, int32_t nz, float *d_sigma,
                              double *d_mean, double *d_energy, void *stream);

/* Adjoint of the explicit MPM stress solve (single-replica handles).  The map:
 * nsteps explicit MPM steps from the current nodal state with the spins
 * frozen (Sec. "Elastic Deformation"), parameters theta = (C11, C12, C44,
 * Ebar_1..6) -- the cubic constants of the handle and its current mean strain
 * -- and outputs W = sum_p w_p and the per-point field w_p = 1/2 eps_p.C'_p.eps_p
 * = 1/2 sigma_p.S'_p.sigma_p (the one-point zone energy of Eq. 8 read at
 * constant traction) at the final state.
 * hmc_adjoint_forward runs the map (the handle's state advances by nsteps MPM
 * steps), keeping (u, v) every checkpoint_every steps on the device; *W
 * (nullable) and w_field (N doubles, natural order, nullable) receive the
 * outputs.  hmc_adjoint_backward then returns in grad[9] the gradient
 * dL/dtheta of L = gW W + sum_p g_p w_p (g_field: N doubles, nullable = 0) by
 * a reverse sweep that recomputes each checkpoint segment forward; it needs
 * the state that hmc_adjoint_forward left (HMC_ERR_STATE if anything changed
 * the spins, nodal state, mean strain or orientations since).  The adjoint
 * buffers are allocated by the first forward call and kept with the handle. */
hmc_status hmc_adjoint_forward(hmc_handle *h, int32_t nsteps, int32_t checkpoint_every, double *W, double *w_field);
hmc_status hmc_adjoint_backward(hmc_handle *h, double gW, const double *g_field, double *grad);

/* Wait for all work on the handle's stream. */
hmc_status hmc_synchronize(hmc_handle *h);

/* Measured peak fused multiply-add rate of the current device (a measurement utility
 * with no counterpart in the paper): precision HMC_FP32 or HMC_FP64; every thread of a
 * grid of the resident CTAs per SM times the SM count runs eight independent FMA chains
 * for iters x 16 steps; *tflops receives 2 flop per FMA over the best of three timed
 * launches (CUDA events on a private stream).  Allocates and frees a small device buffer;
 * HMC_ERR_ARG for a bad precision, iters outside 1..65536 or NULL tflops, HMC_ERR_CUDA
 * on any CUDA error.  Needs no handle. */
hmc_status hmc_fma_peak(int32_t precision, int32_t iters, double *tflops);

/* Message of the last failed call on h (or of the last failed hmc_create when
 * h is NULL).  Valid until the next call on the same handle. */
const char *hmc_last_error(const hmc_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* HMC_H_ */
