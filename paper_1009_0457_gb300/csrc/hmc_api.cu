// C ABI of libhmc (declared and documented in include/hmc.h): handle lifetime,
// host-side orientation tables in FP64, device buffers, the stream order of
// the Monte Carlo step, and the launch-shape autotuner.  A handle holds a
// batch of replicas (hmc_create makes a batch of one); every kernel of the
// Monte Carlo step runs once per phase over all replicas.  Host code only;
// the kernels live in k_*.cu.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "hmc.h"
#include "hmc_internal.h"
#include "hmc_adjoint.h"

using hmc::DevState;

namespace {

thread_local std::string g_create_error;

// Table 1 constants of the calibration (Sec. "Results") used for the default lambda.
constexpr double kGammaStar = 2.4, kGammaS = 0.45, kL0 = 1.0e-3;

int slot_local_h(int s) { static const int t[8] = {0, 3, 5, 6, 1, 2, 4, 7}; return t[s]; }

// Autotuner results, per batch signature, for the life of the process.
std::mutex g_tune_mutex;
struct TuneResult {
    int mpm_shape, mpm_grid, sweep_cta;
    bool store;
};
std::map<std::string, TuneResult> g_tune_cache;

// Host view of one replica.
struct RepHost {
    hmc_params p{};
    int nbx = 0, nby = 0, nbz = 0;
    long long nblk = 0, N = 0, blk_off = 0;
    int cta_off = 0, ncta = 0;
    double axis[3] = {0, 0, 1};
    double lam = 0, lam_sd_half = 0;
};

}  // namespace

namespace hmc {
// Error text for entry points that take no handle, returned by hmc_last_error(NULL).
void set_unbound_error(const std::string &msg) { g_create_error = msg; }
}  // namespace hmc

struct hmc_handle {
    hmc_params p{};                 // shared parameters (replica 0's copy)
    std::vector<RepHost> reps;
    int R = 1, sel = 0;
    long long nblk_total = 0, N_total = 0, N_max = 0;
    int nctas = 0;
    cudaStream_t stream = nullptr, cap = nullptr;
    bool own_stream = false, oriented = false;
    bool lost = false;    // a sweep returned with its stress copy outstanding: every later call is refused
    int num_sms = 0;
    size_t tsize = 4;
    // device buffers
    uint4 *spins = nullptr;
    uint16_t *stage16 = nullptr;
    void *u[2] = {nullptr, nullptr};
    void *v = nullptr;
    int cur = 0;
    void *sig = nullptr, *ctab = nullptr, *wtab = nullptr, *atab = nullptr;
    float *cubw = nullptr;                // FP32 MPM step: Voigt weights of two crystal axes per orientation
    // 27-point zone (HMC_ELASTIC_ZONE1): trial list, start-of-step spins, element tables, schedule
    uint4 *zone_work = nullptr, *snap = nullptr;
    unsigned *zone_count = nullptr;
    void *ktab = nullptr;
    void *stab = nullptr;                 // compliance rows (constant-strain zone)
    uint16_t *zone_sched = nullptr;
    int zone_nsched = 0, zone_grid = 1, zone_scatter_off = 0;
    // grain count: union-find parents of the largest replica, root count and error word
    unsigned *cc_parent = nullptr;
    unsigned long long *cc_count = nullptr;
    unsigned long long *thr = nullptr, *counts = nullptr, *bins = nullptr;
    double *partials = nullptr, *fractions = nullptr;
    int32_t *binmap = nullptr;
    int bins_cap = 0;
    DevState *st = nullptr;               // R device states
    hmc::Replica *d_reps = nullptr;       // R descriptors
    hmc::Replica rep0{};                  // host copy of descriptor 0 (kernel argument of one-replica sweeps)
    int *d_cta_rep = nullptr;             // replica of every sweep / stress CTA
    hmc::MpmSched *d_sched = nullptr;     // R + 1 MPM schedules for the chosen shape
    // MPM launch configuration (autotuned)
    int mpm_shape = hmc::MPM_16x16, mpm_grid = 1;
    long long mpm_total = 0;
    bool tuned = false;
    int sweep_cta = 256;                  // sweep threads per CTA (tuned)
    double *plain_sig = nullptr, *plain_f = nullptr;   // the plain FP64 step's point stresses, cell forces
    bool store_eff = true;                // the step's stress pass stores the stress for the sweeps (tuned
                                          // when store_stress = 2)
    // derived scalars
    double dt = 0, damping = 0, S11 = 0, S12 = 0, S44 = 0;
    // host tables (FP64)
    std::vector<double> A, Cv, Sv;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    std::string err;
    // adjoint of the MPM solve (single replica; allocated by the first hmc_adjoint_forward)
    struct {
        int steps = 0, ck = 0, nseg = 0, nctas = 0;
        bool have_forward = false;
        long long state_version = -1;
        int rtab_version = -1;
        void *rtab = nullptr, *lam = nullptr, *ubar = nullptr, *tmp = nullptr, *vtmp = nullptr, *seg = nullptr;
        void *ck_u = nullptr, *ck_v = nullptr, *w = nullptr, *g = nullptr, *fcell = nullptr;
        double *partials = nullptr, *grad = nullptr;
        hmc::Replica *reps0 = nullptr;   // descriptors whose state has Ebar = 0
        DevState *st0 = nullptr;
        double ebar[6] = {0, 0, 0, 0, 0, 0};
    } adj;
    long long state_version = 0;   // advanced by every call that changes spins, nodal state or Ebar
    int orient_version = 0;
};

namespace {

hmc_status fail(hmc_handle *h, hmc_status s, const std::string &msg) {
    if (h)
        h->err = msg;
    else
        g_create_error = msg;
    return s;
}

hmc_status cuda_fail(hmc_handle *h, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(h, e == cudaErrorMemoryAllocation ? HMC_ERR_OOM : HMC_ERR_CUDA, m);
}

#define HMC_CK(h, call, what)                             \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

// Host-side fault injection for tests of the failure paths (no GPU fault is
// ever produced): HMC_FAULT=alloc fails the next handle creation before any
// CUDA call, =launch fails the next MPM / Monte Carlo launch sequence before it
// is enqueued, =nan writes a NaN into the first nodal displacement before the
// next stress pass, so the FP64 reductions report HMC_ERR_NONFINITE, and
// =sweep_wait makes the stored-stress sweeps enqueued from then on skip their
// stress copy, so that each CTA's bounded wait for it runs out (1 s) and the
// sweep reports HMC_ERR_TIMEOUT.
bool fault(const char *what) {
    const char *f = std::getenv("HMC_FAULT");
    return f && std::strcmp(f, what) == 0;
}

RepHost &selr(hmc_handle *h) { return h->reps[h->sel]; }
DevState *sel_st(hmc_handle *h) { return h->st + h->sel; }
size_t node_bytes(const hmc_handle *h) { return h->tsize * 3 * (size_t)h->nblk_total; }

// ---- FP64 host tables -------------------------------------------------------

// A = Rz(phi) Ry(theta) Rz(psi) written out in closed form (Eq. 18, z-y-z angles).
void euler_zyz(double phi, double theta, double psi, double *A) {
    const double cf = std::cos(phi), sf = std::sin(phi), ct = std::cos(theta), st = std::sin(theta);
    const double cp = std::cos(psi), sp = std::sin(psi);
    A[0] = cf * ct * cp - sf * sp; A[1] = -cf * ct * sp - sf * cp; A[2] = cf * st;
    A[3] = sf * ct * cp + cf * sp; A[4] = -sf * ct * sp + cf * cp; A[5] = sf * st;
    A[6] = -st * cp;               A[7] = st * sp;                 A[8] = ct;
}

const int VI[6] = {0, 1, 2, 1, 0, 0}, VJ[6] = {0, 1, 2, 2, 2, 1};

// Bond matrices of a rotation (Bond 1943): stress sigma' = M sigma, engineering
// strain eps' = Ns eps; then C' = M C M^T and S' = Ns S Ns^T (Eq. 17 in 6x6 form).
void bond(const double *A, double *M, double *Ns) {
    for (int I = 0; I < 6; ++I)
        for (int J = 0; J < 6; ++J) {
            const int i = VI[I], j = VJ[I], k = VI[J], l = VJ[J];
            const double a = A[3 * i + k] * A[3 * j + l], b = A[3 * i + l] * A[3 * j + k];
            M[6 * I + J] = (k == l) ? a : a + b;
            const double fi = (I < 3) ? 1.0 : 2.0;
            Ns[6 * I + J] = fi * ((k == l) ? a : 0.5 * (a + b));
        }
}

void congruence(const double *M, const double *X, double *out) {  // M X M^T
    double t[36];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double s = 0;
            for (int k = 0; k < 6; ++k) s += M[6 * i + k] * X[6 * k + j];
            t[6 * i + j] = s;
        }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double s = 0;
            for (int k = 0; k < 6; ++k) s += t[6 * i + k] * M[6 * j + k];
            out[6 * i + j] = s;
        }
}

template <typename T>
std::vector<T> pack_ctab(const std::vector<double> &Cv, int Q) {
    std::vector<T> out((size_t)Q * 24, T(0));
    for (int q = 0; q < Q; ++q) {
        int n = 0;
        for (int i = 0; i < 6; ++i)
            for (int j = i; j < 6; ++j) out[(size_t)q * 24 + n++] = (T)Cv[(size_t)q * 36 + 6 * i + j];
    }
    return out;
}

template <typename T>
std::vector<T> pack_wtab(const std::vector<double> &A, int Q) {
    std::vector<T> out((size_t)Q * 20, T(0));
    for (int q = 0; q < Q; ++q)
        for (int m = 0; m < 3; ++m) {
            const double *a = &A[(size_t)q * 9];
            const double a1 = a[0 * 3 + m], a2 = a[1 * 3 + m], a3 = a[2 * 3 + m];
            T *w = &out[(size_t)q * 20 + 6 * m];
            w[0] = (T)(a1 * a1); w[1] = (T)(a2 * a2); w[2] = (T)(a3 * a3);
            w[3] = (T)(2 * a2 * a3); w[4] = (T)(2 * a1 * a3); w[5] = (T)(2 * a1 * a2);
        }
    return out;
}

// the first two crystal axes (columns 0 and 1 of A) of every orientation, padded to 8
template <typename T>
std::vector<T> pack_atab(const std::vector<double> &A, int Q) {
    std::vector<T> out((size_t)Q * 8, T(0));
    for (int q = 0; q < Q; ++q)
        for (int m = 0; m < 2; ++m)
            for (int r = 0; r < 3; ++r) out[(size_t)q * 8 + 3 * m + r] = (T)A[(size_t)q * 9 + r * 3 + m];
    return out;
}

void axis_vectors(const double *n, double *N, double *Nsv) {
    N[0] = n[0] * n[0]; N[1] = n[1] * n[1]; N[2] = n[2] * n[2];
    N[3] = n[1] * n[2]; N[4] = n[0] * n[2]; N[5] = n[0] * n[1];
    for (int i = 0; i < 6; ++i) Nsv[i] = (i < 3) ? N[i] : 2 * N[i];
}

// ---- launches ---------------------------------------------------------------

template <typename T>
hmc::MpmArgs<T> mpm_args(hmc_handle *h, const void *u_in, void *u_out, void *v) {
    hmc::MpmArgs<T> a;
    a.reps = h->d_reps;
    a.sched = h->d_sched;
    a.nrep = h->R;
    a.total = h->mpm_total;
    a.spins = h->spins;
    a.u_in = static_cast<const T *>(u_in);
    a.u_out = static_cast<T *>(u_out);
    a.v = static_cast<T *>(v);
    a.ctab = static_cast<const T *>(h->ctab);
    a.cubw = h->cubw;               // FP32 step: cubic form of Hooke's law
    a.cub[0] = (float)h->p.c12;
    a.cub[1] = (float)(2.0 * h->p.c44);
    a.cub[2] = (float)h->p.c44;
    a.cub[3] = (float)(h->p.c11 - h->p.c12 - 2.0 * h->p.c44);
    a.nq = h->p.n_orient;
    a.dt = (T)h->dt;
    a.dt_over_m = (T)(h->dt / 8.0);  // lumped mass rho * V * sum_p N_I(x_p) = 8 voxels
    a.keep = (T)(1.0 - h->damping);
    a.grid = h->mpm_grid;
    return a;
}

cudaError_t enq_mpm(hmc_handle *h, cudaStream_t s) {
    cudaError_t e;
    if (h->p.precision == HMC_FP32)
        e = hmc::launch_mpm_step<float>(mpm_args<float>(h, h->u[h->cur], h->u[h->cur ^ 1], h->v), h->mpm_shape, s);
    else
        e = hmc::launch_mpm_step<double>(mpm_args<double>(h, h->u[h->cur], h->u[h->cur ^ 1], h->v), h->mpm_shape, s);
    h->cur ^= 1;
    return e;
}

template <typename T>
cudaError_t enqueue_stress(hmc_handle *h, bool store, cudaStream_t s) {
    hmc::StressArgs<T> a;
    a.reps = h->d_reps;
    a.cta_rep = h->d_cta_rep;
    a.spins = h->spins;
    a.u = static_cast<const T *>(h->u[h->cur]);
    a.ctab = static_cast<const T *>(h->ctab);
    a.sig = static_cast<T *>(h->sig);
    a.partials = h->partials;
    a.nctas = h->nctas;
    return hmc::launch_stress<T>(a, store, s);
}

template <typename T>
hmc::SweepArgs<T> sweep_args(hmc_handle *h) {
    hmc::SweepArgs<T> a;
    a.reps = h->d_reps;
    a.cta_rep = h->d_cta_rep;
    a.spins = h->spins;
    a.sig = static_cast<const T *>(h->sig);
    a.atab = static_cast<const T *>(h->atab);
    a.thr = h->thr;
    a.trial = h->p.trial;
    a.nq = h->p.n_orient;
    a.J = (T)h->p.J;
    a.kT = (T)h->p.kT;
    a.nctas = h->nctas;
    a.work = h->zone_work;
    a.count = h->zone_count;
    a.ctab = static_cast<const T *>(h->ctab);
    a.stab = static_cast<const T *>(h->stab);
    a.u = static_cast<const T *>(h->u[h->cur]);
    a.skip_copy = fault("sweep_wait") ? 1 : 0;
    a.nrep = h->R;
    a.cta = h->sweep_cta;
    a.margin = nullptr;
    a.rep0 = h->rep0;
    hmc::philox_round_keys(h->rep0.key0, h->rep0.key1, a.rkey);
    return a;
}

template <typename T>
cudaError_t enqueue_sweep(hmc_handle *h, int colour, cudaStream_t s) {
    hmc::SweepArgs<T> a = sweep_args<T>(h);
    const bool point = h->p.elastic == HMC_ELASTIC_TRACTION || h->p.elastic == HMC_ELASTIC_STRAIN;
    if (h->p.elastic != HMC_ELASTIC_ZONE1) {
        const int mode = h->p.elastic == HMC_ELASTIC_TRACTION ? hmc::SWEEP_POINT
                         : h->p.elastic == HMC_ELASTIC_STRAIN ? hmc::SWEEP_STRAIN
                                                              : hmc::SWEEP_POTTS;
        const bool recompute = point && !h->store_eff;
        return hmc::launch_sweep<T>(a, colour, mode, recompute, s);
    }
    // 27-point zone: list the trials, copy the spins as they are at the start of the half step,
    // then decide every listed trial against that copy
    cudaError_t e;
    if ((e = cudaMemsetAsync(h->zone_count, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
    if ((e = hmc::launch_sweep<T>(a, colour, hmc::SWEEP_ZONE_LIST, false, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(h->snap, h->spins, sizeof(uint4) * (size_t)h->nblk_total, cudaMemcpyDeviceToDevice,
                             s)) != cudaSuccess)
        return e;
    hmc::ZoneArgs<T> z;
    z.reps = h->d_reps;
    z.snap = h->snap;
    z.spins = h->spins;
    z.u = static_cast<const T *>(h->u[h->cur]);
    z.ctab = static_cast<const T *>(h->ctab);
    z.ktab = static_cast<const T *>(h->ktab);
    z.work = h->zone_work;
    z.count = h->zone_count;
    z.thr = h->thr;
    z.sched = h->zone_sched;
    z.scatter = h->zone_sched + h->zone_scatter_off;
    z.nsched = h->zone_nsched;
    z.J = (T)h->p.J;
    z.kT = (T)h->p.kT;
    return hmc::launch_zone<T>(z, h->zone_grid, s);
}

// store: write every point's stress (the explicit stress pass, and the Monte Carlo step when the
// sweeps read it); otherwise only the reductions of the end of the step
cudaError_t enq_stress(hmc_handle *h, bool store, cudaStream_t s) {
    return h->p.precision == HMC_FP32 ? enqueue_stress<float>(h, store, s) : enqueue_stress<double>(h, store, s);
}
cudaError_t enq_sweep(hmc_handle *h, int c, cudaStream_t s) {
    return h->p.precision == HMC_FP32 ? enqueue_sweep<float>(h, c, s) : enqueue_sweep<double>(h, c, s);
}

// The sweeps read the stored stress only with a point-zone elastic term and store_stress set.
bool sweeps_read_stress(const hmc_handle *h) {
    return (h->p.elastic == HMC_ELASTIC_TRACTION || h->p.elastic == HMC_ELASTIC_STRAIN) && h->store_eff;
}

// One Monte Carlo step of every replica on stream s (also used while capturing the graph).
cudaError_t enqueue_mcs(hmc_handle *h, cudaStream_t s) {
    cudaError_t e;
    for (int k = 0; k < h->p.mpm_steps_per_mcs; ++k)
        if ((e = enq_mpm(h, s)) != cudaSuccess) return e;
    if ((e = enq_stress(h, sweeps_read_stress(h), s)) != cudaSuccess) return e;
    if ((e = enq_sweep(h, 0, s)) != cudaSuccess) return e;
    if ((e = enq_sweep(h, 1, s)) != cudaSuccess) return e;
    return hmc::launch_end_mcs(h->d_reps, h->R, h->partials, h->nctas, 1, 1, s);
}

cudaError_t reset_accepted(hmc_handle *h) {
    return cudaMemset2DAsync(&h->st->accepted, sizeof(DevState), 0, sizeof(unsigned long long), h->R, h->stream);
}

hmc_status read_accepted(hmc_handle *h, int64_t *acc) {
    std::vector<unsigned long long> a(h->R);
    HMC_CK(h, cudaMemcpy2DAsync(a.data(), sizeof(unsigned long long), &h->st->accepted, sizeof(DevState),
                                sizeof(unsigned long long), h->R, cudaMemcpyDeviceToHost, h->stream),
           "download");
    std::vector<int32_t> bad(h->R);
    HMC_CK(h, cudaMemcpy2DAsync(bad.data(), sizeof(int32_t), &h->st->nonfinite, sizeof(DevState), sizeof(int32_t),
                                h->R, cudaMemcpyDeviceToHost, h->stream),
           "download");
    std::vector<int32_t> late(h->R);
    HMC_CK(h, cudaMemcpy2DAsync(late.data(), sizeof(int32_t), &h->st->wait_timeout, sizeof(DevState),
                                sizeof(int32_t), h->R, cudaMemcpyDeviceToHost, h->stream),
           "download");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    int64_t s = 0;
    for (auto x : a) s += (int64_t)x;
    *acc = s;
    for (int r = 0; r < h->R; ++r)
        if (late[r] == 2) {
            h->lost = true;
            return fail(h, HMC_ERR_TIMEOUT, "a sweep's stress copy never completed in replica " + std::to_string(r) +
                                                "; shared memory of later kernels may have been overwritten, so the "
                                                "handle refuses every further call: destroy it");
        }
    for (int r = 0; r < h->R; ++r)
        if (late[r]) {
            // reported once: the sweep that gave up changed nothing, and later sweeps start clean
            HMC_CK(h, cudaMemset2DAsync(&h->st->wait_timeout, sizeof(DevState), 0, sizeof(int32_t), h->R, h->stream),
                   "memset");
            return fail(h, HMC_ERR_TIMEOUT, "a sweep's stress copy did not complete in replica " + std::to_string(r));
        }
    for (int r = 0; r < h->R; ++r)
        if (bad[r]) return fail(h, HMC_ERR_NONFINITE, "non-finite stress or energy in replica " + std::to_string(r));
    return HMC_OK;
}

hmc_status need_oriented(hmc_handle *h) {
    if (!h) return HMC_ERR_ARG;
    if (h->lost) return fail(h, HMC_ERR_STATE, "a sweep returned with its stress copy outstanding; destroy the handle");
    if (!h->oriented) return fail(h, HMC_ERR_STATE, "hmc_set_orientations has not been called");
    return HMC_OK;
}

// Copy one replica's natural-order spin field to the device, check every index
// < Q there (the replica's field is untouched if one is not), then pack it.
hmc_status upload_spins(hmc_handle *h, int r, const uint16_t *spins) {
    RepHost &R = h->reps[r];
    int bad = 0;
    HMC_CK(h, cudaMemcpyAsync(h->stage16, spins, sizeof(uint16_t) * R.N, cudaMemcpyHostToDevice, h->stream),
           "spin upload");
    HMC_CK(h, cudaMemsetAsync(&h->st[r].bad_spin, 0, sizeof(int32_t), h->stream), "memset");
    HMC_CK(h, hmc::launch_check_spins(h->stage16, R.N, h->p.n_orient, h->st + r, h->stream), "spin check");
    HMC_CK(h, cudaMemcpyAsync(&bad, &h->st[r].bad_spin, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream),
           "download");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    if (bad) {
        for (long long i = 0; i < R.N; ++i)
            if (spins[i] >= (uint32_t)h->p.n_orient)
                return fail(h, HMC_ERR_ARG, "spin value >= n_orient at site " + std::to_string(i) +
                                                (h->R > 1 ? " of replica " + std::to_string(r) : ""));
        return fail(h, HMC_ERR_ARG, "spin value >= n_orient");
    }
    HMC_CK(h, hmc::launch_pack_spins(h->stage16, h->spins + R.blk_off, R.p.nx, R.p.ny, R.p.nz, h->stream),
           "pack spins");
    return HMC_OK;
}

std::string validate(const hmc_params *p) {
    if (!p) return "params is NULL";
    auto even = [](int n) { return n >= 4 && n % 2 == 0; };
    if (!even(p->nx) || !even(p->ny) || !even(p->nz)) return "grid edges must be even and >= 4";
    if ((long long)p->nx * p->ny * p->nz > (1ll << 32) - 1) return "grid larger than 2^32 - 1 sites";
    if (p->n_orient < 1 || p->n_orient > 65535) return "n_orient must be in 1..65535";
    const double vals[] = {p->J, p->kT, p->c11, p->c12, p->c44, p->strain, p->dt, p->damping, p->elastic_scale};
    for (double x : vals)
        if (!std::isfinite(x)) return "non-finite parameter";
    if (p->kT < 0) return "kT must be >= 0";
    if (p->bc != HMC_BC_UNIAXIAL && p->bc != HMC_BC_STRAIN6 && p->bc != HMC_BC_TRACTION) return "bad bc";
    if (!std::isfinite(p->stress)) return "non-finite stress";
    if (p->store_stress < 0 || p->store_stress > 2) return "store_stress must be 0, 1 or 2";
    if (p->elastic != HMC_ELASTIC_OFF && p->elastic != HMC_ELASTIC_TRACTION && p->elastic != HMC_ELASTIC_ZONE1 &&
        p->elastic != HMC_ELASTIC_STRAIN)
        return "bad elastic";
    if (p->elastic == HMC_ELASTIC_ZONE1 && (p->nx < 6 || p->ny < 6 || p->nz < 6))
        return "the 27-point zone needs grid edges >= 6";
    if (p->trial != HMC_TRIAL_NEIGHBOR && p->trial != HMC_TRIAL_UNIFORM_Q) return "bad trial";
    if (p->precision != HMC_FP32 && p->precision != HMC_FP64) return "bad precision";
    if (p->mpm_steps_per_mcs < 0) return "mpm_steps_per_mcs must be >= 0";
    if (p->damping >= 1.0) return "damping must be < 1";
    // cubic stability: C11 - C12 > 0, C11 + 2 C12 > 0, C44 > 0
    if (!(p->c11 - p->c12 > 0 && p->c11 + 2 * p->c12 > 0 && p->c44 > 0)) return "stiffness not positive definite";
    if (p->bc == HMC_BC_UNIAXIAL || p->bc == HMC_BC_TRACTION) {
        const double n2 = p->load_axis[0] * p->load_axis[0] + p->load_axis[1] * p->load_axis[1] +
                          p->load_axis[2] * p->load_axis[2];
        if (!(n2 > 0) || !std::isfinite(n2)) return "load_axis must be a non-zero finite vector";
    }
    for (int i = 0; i < 6; ++i)
        if (!std::isfinite(p->strain6[i])) return "non-finite strain6";
    return "";
}

// Fields every replica of a batch must share.
std::string validate_shared(const hmc_params *a, const hmc_params *b) {
    if (a->n_orient != b->n_orient || a->J != b->J || a->kT != b->kT || a->c11 != b->c11 || a->c12 != b->c12 ||
        a->c44 != b->c44 || a->bc != b->bc || a->elastic != b->elastic || a->trial != b->trial ||
        a->mpm_steps_per_mcs != b->mpm_steps_per_mcs || a->dt != b->dt || a->damping != b->damping ||
        a->precision != b->precision || a->stream != b->stream || a->store_stress != b->store_stress)
        return "replicas of a batch must share n_orient, J, kT, c11, c12, c44, bc, elastic, trial, "
               "mpm_steps_per_mcs, dt, damping, precision, stream and store_stress";
    return "";
}

void free_adjoint(hmc_handle *h) {
    void *bufs[] = {h->adj.rtab, h->adj.lam, h->adj.ubar, h->adj.tmp, h->adj.vtmp, h->adj.seg, h->adj.ck_u,
                    h->adj.ck_v, h->adj.w, h->adj.g, h->adj.fcell, h->adj.partials, h->adj.grad, h->adj.reps0,
                    h->adj.st0};
    for (void *b : bufs)
        if (b) cudaFree(b);
    h->adj.rtab = h->adj.lam = h->adj.ubar = h->adj.tmp = h->adj.vtmp = h->adj.seg = nullptr;
    h->adj.ck_u = h->adj.ck_v = h->adj.w = h->adj.g = h->adj.fcell = nullptr;
    h->adj.partials = h->adj.grad = nullptr;
    h->adj.reps0 = nullptr;
    h->adj.st0 = nullptr;
    h->adj.steps = h->adj.ck = h->adj.nseg = 0;
    h->adj.have_forward = false;
    h->adj.rtab_version = -1;
}

void destroy_buffers(hmc_handle *h) {
    free_adjoint(h);
    for (int i = 0; i < 2; ++i)
        if (h->gexec[i]) cudaGraphExecDestroy(h->gexec[i]);
    void *bufs[] = {h->spins, h->stage16, h->u[0], h->u[1], h->v, h->sig, h->ctab, h->cubw, h->wtab, h->atab, h->thr, h->counts,
                    h->bins, h->partials, h->fractions, h->binmap, h->st, h->d_reps, h->d_cta_rep, h->d_sched,
                    h->zone_work, h->snap, h->zone_count, h->ktab, h->zone_sched, h->cc_parent, h->cc_count,
                    h->stab, h->plain_sig, h->plain_f};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

template <typename T>
void unpack_stress_host(const RepHost &R, const std::vector<T> &packed, double *out) {
    const int nx = R.p.nx, ny = R.p.ny;
    for (long long b = 0; b < R.nblk; ++b) {
        const int bx = (int)(b % R.nbx);
        const long long r = b / R.nbx;
        const int by = (int)(r % R.nby), bz = (int)(r / R.nby);
        for (int s = 0; s < 8; ++s) {
            const int L = slot_local_h(s), c = s >> 2, i = s & 3;
            const long long x = 2 * bx + (L & 1), y = 2 * by + ((L >> 1) & 1), z = 2 * bz + (L >> 2);
            const long long p = x + nx * (y + (long long)ny * z);
            for (int k = 0; k < 6; ++k) out[6 * p + k] = (double)packed[4 * ((size_t)(c * 6 + k) * R.nblk + b) + i];
        }
    }
}

template <typename T>
void pack_stress_host(const RepHost &R, const double *in, std::vector<T> &packed) {
    const int nx = R.p.nx, ny = R.p.ny;
    for (long long b = 0; b < R.nblk; ++b) {
        const int bx = (int)(b % R.nbx);
        const long long r = b / R.nbx;
        const int by = (int)(r % R.nby), bz = (int)(r / R.nby);
        for (int s = 0; s < 8; ++s) {
            const int L = slot_local_h(s), c = s >> 2, i = s & 3;
            const long long x = 2 * bx + (L & 1), y = 2 * by + ((L >> 1) & 1), z = 2 * bz + (L >> 2);
            const long long p = x + nx * (y + (long long)ny * z);
            for (int k = 0; k < 6; ++k) packed[4 * ((size_t)(c * 6 + k) * R.nblk + b) + i] = (T)in[6 * p + k];
        }
    }
}

// ---- MPM schedule and autotuner --------------------------------------------

hmc_status upload_sched(hmc_handle *h, int variant) {
    const int shape = variant % hmc::MPM_NSHAPES;
    const int ox = hmc::mpm_shape_cx(shape) - 1, oy = hmc::mpm_shape_cy(shape) - 1;
    std::vector<hmc::MpmSched> sc(h->R + 1);
    long long off = 0;
    for (int r = 0; r < h->R; ++r) {
        const RepHost &R = h->reps[r];
        sc[r].tiles_x = (R.nbx + ox - 1) / ox;
        sc[r].tiles_y = (R.nby + oy - 1) / oy;
        sc[r].plane_off = off;
        off += (long long)sc[r].tiles_x * sc[r].tiles_y * R.nbz;
    }
    sc[h->R].tiles_x = sc[h->R].tiles_y = 0;
    sc[h->R].plane_off = off;
    h->mpm_total = off;
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    HMC_CK(h, cudaMemcpy(h->d_sched, sc.data(), sizeof(hmc::MpmSched) * sc.size(), cudaMemcpyHostToDevice),
           "schedule upload");
    return HMC_OK;
}

// Persistent MPM grid: resident CTAs per SM (at most per_sm_limit when positive) times the
// SMs, and no more CTAs than leave min_planes work items (planes) to each.  Every CTA pays
// one plane of restart for its range, so small grids trade that for parallelism.
int grid_for_shape(hmc_handle *h, int shape, int per_sm_limit, int min_planes = 4) {
    int per_sm = h->p.precision == HMC_FP32 ? hmc::mpm_per_sm<float>(shape, h->p.n_orient)
                                            : hmc::mpm_per_sm<double>(shape, h->p.n_orient);
    if (per_sm_limit > 0 && per_sm > per_sm_limit) per_sm = per_sm_limit;
    long long g = (long long)per_sm * h->num_sms;
    const long long cap = (h->mpm_total + min_planes - 1) / min_planes;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

std::string tune_signature(const hmc_handle *h) {
    std::string s = std::to_string(h->p.precision) + ":" + std::to_string(h->num_sms) + ":" +
                    std::to_string(h->p.elastic) + ":" + std::to_string(h->p.store_stress) + ":" +
                    std::to_string(h->p.n_orient);
    for (const auto &R : h->reps)
        s += ":" + std::to_string(R.nbx) + "x" + std::to_string(R.nby) + "x" + std::to_string(R.nbz);
    return s;
}

// Pick the MPM patch shape and persistent-grid size by timing every candidate
// on scratch copies of the nodal state (the simulation state is not touched).
// Every candidate computes bit-identical results: the per-cell arithmetic
// (explicitly rounded, in one order, paired or not) and the order of each
// node's force sum do not depend on the variant.
hmc_status tune_mpm(hmc_handle *h, bool enabled, int &best_shape, int &best_grid) {
    hmc_status s = HMC_OK;
    best_shape = hmc::MPM_16x16;
    if ((s = upload_sched(h, best_shape)) != HMC_OK) return s;
    best_grid = grid_for_shape(h, best_shape, 0);
    if (!enabled) return HMC_OK;
    const size_t nb = node_bytes(h);
    void *uo = nullptr, *vs = nullptr;
    HMC_CK(h, cudaMalloc(&uo, nb), "autotune scratch");
    if (cudaMalloc(&vs, nb) != cudaSuccess) {
        cudaFree(uo);
        return fail(h, HMC_ERR_OOM, "autotune scratch");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    cudaError_t err = cudaMemcpyAsync(vs, h->v, nb, cudaMemcpyDeviceToDevice, h->stream);
    const int nvariants = hmc::mpm_nvariants(h->p.precision == HMC_FP32);
    for (int shape = 0; shape < nvariants && err == cudaSuccess && s == HMC_OK; ++shape) {
        if ((s = upload_sched(h, shape)) != HMC_OK) break;
        // full occupancy and one CTA per SM with at least four planes per CTA, then (small grids)
        // full occupancy with at least two planes and with at least one
        std::vector<int> tried;
        for (int cand = 0; cand < 4; ++cand) {
            const int grid = grid_for_shape(h, shape, cand == 1 ? 1 : 0, cand < 2 ? 4 : cand == 2 ? 2 : 1);
            if (std::find(tried.begin(), tried.end(), grid) != tried.end()) continue;
            tried.push_back(grid);
            const int saved_grid = h->mpm_grid;
            h->mpm_grid = grid;
            auto launch = [&]() {
                return h->p.precision == HMC_FP32
                           ? hmc::launch_mpm_step<float>(mpm_args<float>(h, h->u[h->cur], uo, vs), shape, h->stream)
                           : hmc::launch_mpm_step<double>(mpm_args<double>(h, h->u[h->cur], uo, vs), shape,
                                                          h->stream);
            };
            err = launch();
            if (err == cudaSuccess) err = cudaEventRecord(e0, h->stream);
            for (int k = 0; k < 3 && err == cudaSuccess; ++k) err = launch();
            if (err == cudaSuccess) err = cudaEventRecord(e1, h->stream);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float ms = 0;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            h->mpm_grid = saved_grid;
            if (err == cudaSuccess && ms < best) {
                best = ms;
                best_shape = shape;
                best_grid = grid;
            }
            if (err != cudaSuccess) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(h->stream);
    cudaFree(uo);
    cudaFree(vs);
    if (s != HMC_OK) return s;
    if (err != cudaSuccess) return cuda_fail(h, err, "autotune");
    return upload_sched(h, best_shape);
}

// Pick the sweep CTA size (256 threads per 256-block tile, or the tile split over two
// CTAs of 128) and, with store_stress = 2 and the constant-traction point zone,
// whether a Monte Carlo step stores every point's stress for the sweeps or the
// sweeps recompute each trial site's stress from the nodal displacement.  Every
// candidate gives the same decisions (the stored and recomputed forms evaluate the
// same rounded arithmetic; the CTA size only changes which CTA decides a site), so
// the choice never changes a result.  Each candidate is timed as a step runs it --
// the stress pass (storing or not), the red and the black half sweep -- on a scratch
// copy of the spins, with the stress written to scratch memory, so the simulation
// state is not touched (only the acceptance counter, which every sweep resets).
hmc_status tune_sweeps(hmc_handle *h, bool enabled) {
    const bool point = h->p.elastic == HMC_ELASTIC_TRACTION || h->p.elastic == HMC_ELASTIC_STRAIN;
    h->sweep_cta = 256;
    h->store_eff = h->p.store_stress != 0;
    if (!(point || h->p.elastic == HMC_ELASTIC_OFF)) return HMC_OK;   // the zone form lists trials
    const bool auto_store = h->p.store_stress == 2 && h->p.elastic == HMC_ELASTIC_TRACTION;
    if (!enabled || h->nblk_total < 256) return HMC_OK;
    const size_t nsp = sizeof(uint4) * (size_t)h->nblk_total;
    const size_t nsig = (size_t)48 * h->tsize * (size_t)h->nblk_total;
    void *spn = nullptr, *sig = nullptr, *part = nullptr;
    HMC_CK(h, cudaMalloc(&spn, nsp), "autotune scratch");
    cudaError_t err = cudaMalloc(&sig, point ? nsig : 16);
    if (err == cudaSuccess) err = cudaMalloc(&part, sizeof(double) * 7 * (size_t)h->nctas);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    float best = 1e30f;
    int best_cta = 256;
    bool best_store = h->store_eff;
    for (int store = 1; store >= 0 && err == cudaSuccess; --store) {
        if (!auto_store && store != (int)h->store_eff) continue;
        for (int cta : {256, 128}) {
            if (cta == 128 && point && !store) continue;   // the recomputing form has one CTA size
            float t = 1e30f;
            for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
                err = cudaMemcpyAsync(spn, h->spins, nsp, cudaMemcpyDeviceToDevice, h->stream);
                if (err == cudaSuccess) err = cudaEventRecord(e0, h->stream);
                if (point && err == cudaSuccess) {
                    auto stress = [&](auto tag) {
                        using T = decltype(tag);
                        hmc::StressArgs<T> a;
                        a.reps = h->d_reps;
                        a.cta_rep = h->d_cta_rep;
                        a.spins = static_cast<const uint4 *>(spn);
                        a.u = static_cast<const T *>(h->u[h->cur]);
                        a.ctab = static_cast<const T *>(h->ctab);
                        a.sig = static_cast<T *>(sig);
                        a.partials = static_cast<double *>(part);
                        a.nctas = h->nctas;
                        return hmc::launch_stress<T>(a, store != 0, h->stream);
                    };
                    err = h->p.precision == HMC_FP32 ? stress(float()) : stress(double());
                }
                for (int c = 0; c < 2 && err == cudaSuccess; ++c) {
                    auto sweep = [&](auto tag) {
                        using T = decltype(tag);
                        hmc::SweepArgs<T> a = sweep_args<T>(h);
                        a.spins = static_cast<uint4 *>(spn);
                        a.sig = static_cast<const T *>(sig);
                        a.cta = cta;
                        a.skip_copy = 0;
                        const int mode = h->p.elastic == HMC_ELASTIC_TRACTION ? hmc::SWEEP_POINT
                                         : h->p.elastic == HMC_ELASTIC_STRAIN ? hmc::SWEEP_STRAIN
                                                                              : hmc::SWEEP_POTTS;
                        return hmc::launch_sweep<T>(a, c, mode, point && !store, h->stream);
                    };
                    err = h->p.precision == HMC_FP32 ? sweep(float()) : sweep(double());
                }
                if (err == cudaSuccess) err = cudaEventRecord(e1, h->stream);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                float ms = 0;
                if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
                if (err == cudaSuccess && ms < t) t = ms;
            }
            if (err == cudaSuccess && t < best) {
                best = t;
                best_cta = cta;
                best_store = store != 0;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(h->stream);
    cudaFree(spn);
    cudaFree(sig);
    cudaFree(part);
    if (err != cudaSuccess) return cuda_fail(h, err, "sweep autotune");
    h->sweep_cta = best_cta;
    h->store_eff = best_store;
    return HMC_OK;
}

// The tuned launch configuration, once per handle at its first MPM use (before any graph
// capture): cached per batch signature for the life of the process.  HMC_AUTOTUNE=0 keeps
// the defaults (16x16 MPM patches, 256-thread sweep CTAs, stored stress in auto mode);
// HMC_MPM_SHAPE=<variant> and HMC_SWEEP_CTA=128|256 force a choice.
hmc_status ensure_tuned(hmc_handle *h) {
    if (h->tuned) return HMC_OK;
    hmc_status s = HMC_OK;
    const char *env = std::getenv("HMC_AUTOTUNE");
    const bool enabled = !(env && env[0] == '0');
    const char *forced = std::getenv("HMC_MPM_SHAPE");
    const char *forced_cta = std::getenv("HMC_SWEEP_CTA");
    const int nvar = hmc::mpm_nvariants(h->p.precision == HMC_FP32);
    const bool force_mpm = forced && forced[0] >= '0' && forced[0] < '0' + nvar && forced[1] == 0;
    const bool force_cta = forced_cta && (std::string(forced_cta) == "128" || std::string(forced_cta) == "256");
    const std::string sig = tune_signature(h);
    if (!force_mpm && !force_cta) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(sig);
        if (it != g_tune_cache.end()) {
            if ((s = upload_sched(h, it->second.mpm_shape)) != HMC_OK) return s;
            h->mpm_shape = it->second.mpm_shape;
            h->mpm_grid = it->second.mpm_grid;
            h->sweep_cta = it->second.sweep_cta;
            h->store_eff = it->second.store;
            h->tuned = true;
            return HMC_OK;
        }
    }
    int shape = 0, grid = 1;
    if (force_mpm) {
        shape = forced[0] - '0';
        if ((s = upload_sched(h, shape)) != HMC_OK) return s;
        grid = grid_for_shape(h, shape, 0);
    } else if ((s = tune_mpm(h, enabled, shape, grid)) != HMC_OK) {
        return s;
    }
    h->mpm_shape = shape;
    h->mpm_grid = grid;
    if ((s = tune_sweeps(h, enabled && !force_cta)) != HMC_OK) return s;
    if (force_cta) h->sweep_cta = std::atoi(forced_cta);
    h->tuned = true;
    if (!force_mpm && !force_cta) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[sig] = TuneResult{h->mpm_shape, h->mpm_grid, h->sweep_cta, h->store_eff};
    }
    return HMC_OK;
}

hmc_status read_stats(hmc_handle *h, double *mean, double *energy) {
    DevState st;
    HMC_CK(h, cudaMemcpyAsync(&st, sel_st(h), sizeof(st), cudaMemcpyDeviceToHost, h->stream), "state download");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    if (st.wait_timeout == 2) {
        h->lost = true;
        return fail(h, HMC_ERR_TIMEOUT, "a sweep's stress copy never completed; the handle refuses every further call");
    }
    if (st.wait_timeout) {
        HMC_CK(h, cudaMemsetAsync(&sel_st(h)->wait_timeout, 0, sizeof(int32_t), h->stream), "memset");
        return fail(h, HMC_ERR_TIMEOUT, "a sweep's stress copy did not complete");
    }
    if (st.nonfinite) return fail(h, HMC_ERR_NONFINITE, "non-finite stress or energy");
    if (mean)
        for (int i = 0; i < 6; ++i) mean[i] = st.mean_sigma[i];
    if (energy) *energy = st.energy;
    return HMC_OK;
}

hmc_status nodal_io(hmc_handle *h, void *dev_base, double *host, bool to_host) {
    const RepHost &R = selr(h);
    const size_t n = 3 * (size_t)R.nblk;
    char *dev = static_cast<char *>(dev_base) + h->tsize * 3 * (size_t)R.blk_off;
    if (h->p.precision == HMC_FP64) {
        if (to_host)
            HMC_CK(h, cudaMemcpyAsync(host, dev, n * 8, cudaMemcpyDeviceToHost, h->stream), "download");
        else
            HMC_CK(h, cudaMemcpyAsync(dev, host, n * 8, cudaMemcpyHostToDevice, h->stream), "upload");
        HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
        return HMC_OK;
    }
    std::vector<float> t(n);
    if (to_host) {
        HMC_CK(h, cudaMemcpyAsync(t.data(), dev, n * 4, cudaMemcpyDeviceToHost, h->stream), "download");
        HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
        for (size_t i = 0; i < n; ++i) host[i] = t[i];
    } else {
        for (size_t i = 0; i < n; ++i) t[i] = (float)host[i];
        HMC_CK(h, cudaMemcpyAsync(dev, t.data(), n * 4, cudaMemcpyHostToDevice, h->stream), "upload");
        HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    }
    return HMC_OK;
}

struct StateHeader {
    char magic[8];
    int32_t nx, ny, nz, precision;
    uint32_t mcs, pad;
    double ebar[6];
};

}  // namespace

extern "C" {

void hmc_default_params(hmc_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->nx = p->ny = p->nz = 32;
    p->n_orient = 64;
    p->J = 1.0;
    p->kT = 0.7;
    p->c11 = 246.5; p->c12 = 147.3; p->c44 = 124.7;
    p->bc = HMC_BC_UNIAXIAL;
    p->load_axis[2] = 1.0;
    p->strain = 1e-3;
    p->elastic_scale = -1.0;
    p->elastic = HMC_ELASTIC_TRACTION;
    p->store_stress = 1;
    p->trial = HMC_TRIAL_NEIGHBOR;
    p->mpm_steps_per_mcs = 50;
    p->dt = -1.0;
    p->damping = -1.0;
    p->precision = HMC_FP32;
    p->seed = 1;
    p->replica = 0;
    p->stream = nullptr;
}

hmc_status hmc_create_batch(const hmc_params *params, int32_t n_replicas, hmc_handle **out) {
    if (!out) return fail(nullptr, HMC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!params || n_replicas < 1) return fail(nullptr, HMC_ERR_ARG, "need params for at least one replica");
    if (fault("alloc")) return fail(nullptr, HMC_ERR_OOM, "injected allocation failure (HMC_FAULT=alloc)");
    for (int r = 0; r < n_replicas; ++r) {
        std::string msg = validate(params + r);
        if (msg.empty() && r > 0) msg = validate_shared(params, params + r);
        if (!msg.empty())
            return fail(nullptr, HMC_ERR_ARG, n_replicas > 1 ? "replica " + std::to_string(r) + ": " + msg : msg);
    }
    hmc_handle *h = new (std::nothrow) hmc_handle();
    if (!h) return fail(nullptr, HMC_ERR_OOM, "host allocation failed");
    const hmc_params *p = params;
    h->p = *p;
    h->store_eff = p->store_stress != 0;   // auto (2) starts stored; the tuner may switch it
    h->R = n_replicas;
    h->tsize = p->precision == HMC_FP32 ? 4 : 8;
    const double lam_max = std::fmax(std::fmax(p->c11 + 2 * p->c12, p->c11 - p->c12), 2 * p->c44);
    h->dt = p->dt > 0 ? p->dt : 0.5 * 2.0 / std::sqrt(lam_max);
    h->damping = p->damping >= 0 ? p->damping : 0.05;
    const double dd = (p->c11 - p->c12) * (p->c11 + 2 * p->c12);
    h->S11 = (p->c11 + p->c12) / dd;
    h->S12 = -p->c12 / dd;
    h->S44 = 1.0 / p->c44;
    h->reps.resize(n_replicas);
    long long blk = 0;
    int cta = 0;
    for (int r = 0; r < n_replicas; ++r) {
        RepHost &R = h->reps[r];
        R.p = params[r];
        R.nbx = R.p.nx / 2; R.nby = R.p.ny / 2; R.nbz = R.p.nz / 2;
        R.nblk = (long long)R.nbx * R.nby * R.nbz;
        R.N = 8 * R.nblk;
        R.blk_off = blk;
        blk += R.nblk;
        R.ncta = (int)((R.nblk + hmc::BLOCK_THREADS - 1) / hmc::BLOCK_THREADS);
        R.cta_off = cta;
        cta += R.ncta;
        const int K = std::max(R.p.nx, std::max(R.p.ny, R.p.nz));
        R.lam = R.p.elastic_scale >= 0 ? R.p.elastic_scale : 1e9 * (1.0 / K) * kL0 * kGammaStar / (2.0 * kGammaS);
        R.lam_sd_half = 0.5 * R.lam * (h->S11 - h->S12 - 0.5 * h->S44);
        if (R.p.bc == HMC_BC_UNIAXIAL || R.p.bc == HMC_BC_TRACTION) {
            const double n = std::sqrt(R.p.load_axis[0] * R.p.load_axis[0] + R.p.load_axis[1] * R.p.load_axis[1] +
                                       R.p.load_axis[2] * R.p.load_axis[2]);
            for (int i = 0; i < 3; ++i) R.axis[i] = R.p.load_axis[i] / n;
        }
        h->N_total += R.N;
        h->N_max = std::max(h->N_max, R.N);
    }
    h->nblk_total = blk;
    h->nctas = cta;

    auto bail = [&](hmc_status s) {
        g_create_error = h->err;
        destroy_buffers(h);
        delete h;
        return s;
    };
    cudaError_t e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return bail(cuda_fail(h, e, "cudaGetDevice"));
    if ((e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return bail(cuda_fail(h, e, "device attribute"));
    if (p->stream) {
        h->stream = static_cast<cudaStream_t>(p->stream);
    } else {
        if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(cuda_fail(h, e, "stream create"));
        h->own_stream = true;
    }
    if ((e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(cuda_fail(h, e, "capture stream create"));
    if ((e = hmc::mpm_prepare()) != cudaSuccess) return bail(cuda_fail(h, e, "MPM kernel attribute"));
    if ((e = hmc::sweep_prepare()) != cudaSuccess) return bail(cuda_fail(h, e, "sweep kernel attribute"));
    struct Alloc { void **ptr; size_t bytes; const char *what; };
    const size_t nodes_b = node_bytes(h);
    Alloc allocs[] = {
        {(void **)&h->spins, sizeof(uint4) * (size_t)h->nblk_total, "spins"},
        {(void **)&h->stage16, sizeof(uint16_t) * (size_t)h->N_max, "spin staging"},
        {&h->u[0], nodes_b, "u0"}, {&h->u[1], nodes_b, "u1"}, {&h->v, nodes_b, "v"},
        {&h->sig, h->tsize * 48 * (size_t)h->nblk_total, "stress"},
        {&h->ctab, h->tsize * 24 * (size_t)p->n_orient, "stiffness table"},
        {(void **)&h->cubw, sizeof(float) * 12 * (size_t)p->n_orient, "cubic axis table"},
        {&h->wtab, h->tsize * 20 * (size_t)p->n_orient, "axis weight table"},
        {&h->atab, h->tsize * 8 * (size_t)p->n_orient, "axis table"},
        {(void **)&h->thr, sizeof(unsigned long long) * 8, "threshold table"},
        {(void **)&h->counts, sizeof(unsigned long long) * (size_t)p->n_orient, "orientation counts"},
        {(void **)&h->partials, sizeof(double) * (7 * (size_t)h->nctas + hmc::end_scratch_doubles(h->R)), "partials"},
        {(void **)&h->st, sizeof(DevState) * (size_t)h->R, "device state"},
        {(void **)&h->d_reps, sizeof(hmc::Replica) * (size_t)h->R, "replica table"},
        {(void **)&h->d_cta_rep, sizeof(int) * (size_t)h->nctas, "CTA table"},
        {(void **)&h->d_sched, sizeof(hmc::MpmSched) * (size_t)(h->R + 1), "MPM schedule"},
    };
    for (auto &a : allocs) {
        if ((e = cudaMalloc(a.ptr, a.bytes)) != cudaSuccess) return bail(cuda_fail(h, e, a.what));
    }
    // integer Metropolis thresholds for an integer bond-energy change k (Eq. 5)
    unsigned long long thr[8];
    for (int k = 0; k < 8; ++k) {
        double t;
        if (k <= 0)
            t = 4294967296.0;
        else if (!(p->kT > 0.0))
            t = 0.0;
        else
            t = std::ceil(std::exp(-(double)k * p->J / p->kT) * 4294967296.0 - 0.5);
        thr[k] = (unsigned long long)t;
    }
    if ((e = cudaMemcpy(h->thr, thr, sizeof(thr), cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(cuda_fail(h, e, "threshold upload"));
    std::vector<DevState> st(h->R);
    std::vector<hmc::Replica> rd(h->R);
    std::vector<int> ctarep(h->nctas);
    for (int r = 0; r < h->R; ++r) {
        const RepHost &R = h->reps[r];
        std::memset(&st[r], 0, sizeof(DevState));
        st[r].bc = R.p.bc;
        std::memset(&rd[r], 0, sizeof(hmc::Replica));
        rd[r].nx = R.p.nx; rd[r].ny = R.p.ny; rd[r].nz = R.p.nz;
        rd[r].nbx = R.nbx; rd[r].nby = R.nby; rd[r].nbz = R.nbz;
        rd[r].nblk = (int)R.nblk;
        rd[r].cta_off = R.cta_off;
        rd[r].ncta = R.ncta;
        rd[r].blk_off = R.blk_off;
        rd[r].key0 = (uint32_t)(R.p.seed & 0xffffffffull);
        rd[r].key1 = (uint32_t)(R.p.seed >> 32);
        rd[r].replica = R.p.replica;
        rd[r].lam_sd_half = R.lam_sd_half;
        rd[r].lam = R.lam;
        rd[r].lam_sd_half_f = (float)R.lam_sd_half;
        rd[r].lam_f = (float)R.lam;
        rd[r].st = h->st + r;
        rd[r].divx = hmc::make_udiv((uint32_t)R.nbx);
        rd[r].divy = hmc::make_udiv((uint32_t)R.nby);
        for (int c = 0; c < R.ncta; ++c) ctarep[R.cta_off + c] = r;
    }
    h->rep0 = rd[0];
    if ((e = cudaMemcpy(h->st, st.data(), sizeof(DevState) * st.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(h->d_reps, rd.data(), sizeof(hmc::Replica) * rd.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(h->d_cta_rep, ctarep.data(), sizeof(int) * ctarep.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
        return bail(cuda_fail(h, e, "descriptor upload"));
    void *zero_ptrs[] = {h->u[0], h->u[1], h->v};
    for (void *z : zero_ptrs)
        if ((e = cudaMemset(z, 0, nodes_b)) != cudaSuccess) return bail(cuda_fail(h, e, "memset"));
    // the end-of-step reduction's arrival counters start at zero
    if ((e = cudaMemset(h->partials, 0, sizeof(double) * (7 * (size_t)h->nctas + hmc::end_scratch_doubles(h->R)))) !=
        cudaSuccess)
        return bail(cuda_fail(h, e, "memset"));
    if (p->elastic == HMC_ELASTIC_STRAIN &&
        (e = cudaMalloc(&h->stab, h->tsize * 24 * (size_t)p->n_orient)) != cudaSuccess)
        return bail(cuda_fail(h, e, "compliance table"));
    if (p->elastic == HMC_ELASTIC_ZONE1) {
        std::vector<uint16_t> zs = hmc::zone_schedule();
        if (zs.empty()) return bail(fail(h, HMC_ERR_CUDA, "zone schedule does not fit"));
        h->zone_nsched = (int)zs.size();
        const std::vector<uint16_t> scat = hmc::zone_scatter_table(zs);
        zs.resize((zs.size() + 7) & ~size_t(7), 0);   // the scatter table starts 16-byte aligned
        h->zone_scatter_off = (int)zs.size();
        zs.insert(zs.end(), scat.begin(), scat.end());
        Alloc za[] = {
            {(void **)&h->zone_work, sizeof(uint4) * 4 * (size_t)h->nblk_total, "zone trial list"},
            {(void **)&h->snap, sizeof(uint4) * (size_t)h->nblk_total, "spin copy"},
            {(void **)&h->zone_count, sizeof(unsigned), "zone trial count"},
            {&h->ktab, h->tsize * 8 * 320 * (size_t)p->n_orient, "zone element tables"},
            {(void **)&h->zone_sched, sizeof(uint16_t) * zs.size(), "zone schedule"},
        };
        for (auto &a : za)
            if ((e = cudaMalloc(a.ptr, a.bytes)) != cudaSuccess) return bail(cuda_fail(h, e, a.what));
        if ((e = cudaMemcpy(h->zone_sched, zs.data(), sizeof(uint16_t) * zs.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            return bail(cuda_fail(h, e, "zone schedule upload"));
        if ((e = hmc::zone_prepare()) != cudaSuccess) return bail(cuda_fail(h, e, "zone kernel attribute"));
        const int per_sm = p->precision == HMC_FP32 ? hmc::zone_per_sm<float>() : hmc::zone_per_sm<double>();
        h->zone_grid = h->num_sms * per_sm;
    }
    hmc_status s = upload_sched(h, h->mpm_shape);
    if (s != HMC_OK) return bail(s);
    h->mpm_grid = grid_for_shape(h, h->mpm_shape, 0);
    *out = h;
    return HMC_OK;
}

hmc_status hmc_create(const hmc_params *p, hmc_handle **out) { return hmc_create_batch(p, 1, out); }

void hmc_destroy(hmc_handle *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    destroy_buffers(h);
    delete h;
}

hmc_status hmc_select_replica(hmc_handle *h, int32_t r) {
    if (!h) return HMC_ERR_ARG;
    if (r < 0 || r >= h->R) return fail(h, HMC_ERR_ARG, "replica index out of range");
    h->sel = r;
    return HMC_OK;
}

hmc_status hmc_get_tuning(hmc_handle *h, int32_t *mpm_shape, int32_t *mpm_grid) {
    if (!h) return HMC_ERR_ARG;
    if (mpm_shape) *mpm_shape = h->mpm_shape;
    if (mpm_grid) *mpm_grid = h->mpm_grid;
    return HMC_OK;
}

hmc_status hmc_get_sweep_tuning(hmc_handle *h, int32_t *sweep_cta, int32_t *stored) {
    if (!h) return HMC_ERR_ARG;
    if (sweep_cta) *sweep_cta = h->sweep_cta;
    if (stored) *stored = h->store_eff ? 1 : 0;
    return HMC_OK;
}

hmc_status hmc_set_orientations(hmc_handle *h, const double *euler, const uint16_t *spins) {
    if (h) ++h->state_version;
    if (!h) return HMC_ERR_ARG;
    if (!euler || !spins) return fail(h, HMC_ERR_ARG, "NULL euler or spins");
    const int Q = h->p.n_orient;
    for (int i = 0; i < 3 * Q; ++i)
        if (!std::isfinite(euler[i])) return fail(h, HMC_ERR_ARG, "non-finite Euler angle");
    for (long long i = 0; i < h->N_total; ++i)
        if (spins[i] >= (uint32_t)Q)
            return fail(h, HMC_ERR_ARG, "spin value >= n_orient at site " + std::to_string(i));
    h->A.assign((size_t)Q * 9, 0.0);
    h->Cv.assign((size_t)Q * 36, 0.0);
    h->Sv.assign((size_t)Q * 36, 0.0);
    double C0[36] = {0}, S0[36] = {0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            C0[6 * i + j] = (i == j) ? h->p.c11 : h->p.c12;
            S0[6 * i + j] = (i == j) ? h->S11 : h->S12;
        }
    for (int i = 3; i < 6; ++i) {
        C0[6 * i + i] = h->p.c44;
        S0[6 * i + i] = h->S44;
    }
    for (int q = 0; q < Q; ++q) {
        double M[36], Ns[36];
        euler_zyz(euler[3 * q], euler[3 * q + 1], euler[3 * q + 2], &h->A[(size_t)q * 9]);
        bond(&h->A[(size_t)q * 9], M, Ns);
        congruence(M, C0, &h->Cv[(size_t)q * 36]);
        congruence(Ns, S0, &h->Sv[(size_t)q * 36]);
    }
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    // per replica: Reuss compliance of its initial volume fractions, initial mean strain
    std::vector<DevState> st(h->R);
    long long site = 0;
    for (int r = 0; r < h->R; ++r) {
        const RepHost &R = h->reps[r];
        std::vector<long long> cnt(Q, 0);
        for (long long i = 0; i < R.N; ++i) cnt[spins[site + i]]++;
        DevState &d = st[r];
        std::memset(&d, 0, sizeof(d));
        for (int q = 0; q < Q; ++q)
            if (cnt[q])
                for (int k = 0; k < 36; ++k) d.sr[k] += (double)cnt[q] / (double)R.N * h->Sv[(size_t)q * 36 + k];
        d.bc = R.p.bc;
        d.eps0 = R.p.strain;
        if (R.p.bc == HMC_BC_UNIAXIAL) {
            axis_vectors(R.axis, d.axN, d.axNs);
            for (int i = 0; i < 6; ++i) {
                double s = 0;
                for (int j = 0; j < 6; ++j) s += d.sr[6 * i + j] * d.axN[j];
                d.axB[i] = s;
            }
            d.axNB = 0;
            for (int i = 0; i < 6; ++i) d.axNB += d.axN[i] * d.axB[i];
            for (int i = 0; i < 6; ++i) d.ebar[i] = R.p.strain / d.axNB * d.axB[i];
        } else if (R.p.bc == HMC_BC_TRACTION) {
            axis_vectors(R.axis, d.axN, d.axNs);
            d.sig0 = R.p.stress;
            for (int i = 0; i < 6; ++i) {
                double e = 0;
                for (int j = 0; j < 6; ++j) e += d.sr[6 * i + j] * d.sig0 * d.axN[j];
                d.ebar[i] = e;
            }
        } else {
            for (int i = 0; i < 6; ++i) d.ebar[i] = R.p.strain6[i];
        }
        for (int i = 0; i < 6; ++i) d.ebar_f[i] = (float)d.ebar[i];
        site += R.N;
    }
    HMC_CK(h, cudaMemcpy(h->st, st.data(), sizeof(DevState) * h->R, cudaMemcpyHostToDevice), "state upload");
    if (h->p.precision == HMC_FP32) {
        auto c = pack_ctab<float>(h->Cv, Q);
        auto w = pack_wtab<float>(h->A, Q);
        auto ax = pack_atab<float>(h->A, Q);
        HMC_CK(h, cudaMemcpy(h->ctab, c.data(), c.size() * sizeof(float), cudaMemcpyHostToDevice), "table upload");
        HMC_CK(h, cudaMemcpy(h->wtab, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice), "table upload");
        HMC_CK(h, cudaMemcpy(h->atab, ax.data(), ax.size() * sizeof(float), cudaMemcpyHostToDevice), "table upload");
        // the FP32 MPM step's cubic form: Voigt weights (x^2, y^2, z^2, yz, xz, xy) of the crystal
        // axes a_0 and a_1 (columns 0 and 1 of A) of every orientation
        std::vector<float> cw((size_t)Q * 12);
        for (int q = 0; q < Q; ++q)
            for (int m = 0; m < 2; ++m) {
                const double *A = &h->A[(size_t)q * 9];
                const double x = A[0 * 3 + m], y = A[1 * 3 + m], z = A[2 * 3 + m];
                float *w = &cw[(size_t)q * 12 + 6 * m];
                w[0] = (float)(x * x); w[1] = (float)(y * y); w[2] = (float)(z * z);
                w[3] = (float)(y * z); w[4] = (float)(x * z); w[5] = (float)(x * y);
            }
        HMC_CK(h, cudaMemcpy(h->cubw, cw.data(), cw.size() * sizeof(float), cudaMemcpyHostToDevice),
               "table upload");
    } else {
        auto c = pack_ctab<double>(h->Cv, Q);
        auto w = pack_wtab<double>(h->A, Q);
        auto ax = pack_atab<double>(h->A, Q);
        HMC_CK(h, cudaMemcpy(h->ctab, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice), "table upload");
        HMC_CK(h, cudaMemcpy(h->wtab, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice), "table upload");
        HMC_CK(h, cudaMemcpy(h->atab, ax.data(), ax.size() * sizeof(double), cudaMemcpyHostToDevice), "table upload");
    }
    if (h->p.elastic == HMC_ELASTIC_STRAIN) {
        if (h->p.precision == HMC_FP32) {
            auto st32 = pack_ctab<float>(h->Sv, Q);
            HMC_CK(h, cudaMemcpy(h->stab, st32.data(), st32.size() * sizeof(float), cudaMemcpyHostToDevice),
                   "table upload");
        } else {
            auto st64 = pack_ctab<double>(h->Sv, Q);
            HMC_CK(h, cudaMemcpy(h->stab, st64.data(), st64.size() * sizeof(double), cudaMemcpyHostToDevice),
                   "table upload");
        }
    }
    if (h->p.elastic == HMC_ELASTIC_ZONE1) {
        std::vector<double> kt;
        hmc::zone_element_tables(h->Cv.data(), Q, kt);
        if (h->p.precision == HMC_FP32) {
            std::vector<float> kf(kt.begin(), kt.end());
            HMC_CK(h, cudaMemcpy(h->ktab, kf.data(), kf.size() * sizeof(float), cudaMemcpyHostToDevice),
                   "zone table upload");
        } else {
            HMC_CK(h, cudaMemcpy(h->ktab, kt.data(), kt.size() * sizeof(double), cudaMemcpyHostToDevice),
                   "zone table upload");
        }
    }
    const size_t nodes_b = node_bytes(h);
    HMC_CK(h, cudaMemsetAsync(h->u[0], 0, nodes_b, h->stream), "memset u");
    HMC_CK(h, cudaMemsetAsync(h->u[1], 0, nodes_b, h->stream), "memset u");
    HMC_CK(h, cudaMemsetAsync(h->v, 0, nodes_b, h->stream), "memset v");
    HMC_CK(h, cudaMemsetAsync(h->sig, 0, h->tsize * 48 * (size_t)h->nblk_total, h->stream), "memset sigma");
    h->cur = 0;
    site = 0;
    for (int r = 0; r < h->R; ++r) {
        hmc_status s = upload_spins(h, r, spins + site);
        if (s != HMC_OK) return s;
        site += h->reps[r].N;
    }
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    h->oriented = true;
    ++h->orient_version;
    return HMC_OK;
}

hmc_status hmc_set_spins(hmc_handle *h, const uint16_t *spins) {
    if (h) ++h->state_version;
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if (!spins) return fail(h, HMC_ERR_ARG, "NULL spins");
    if ((s = upload_spins(h, h->sel, spins)) != HMC_OK) return s;
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    return HMC_OK;
}

namespace {
// Device pointers handed in by the caller: memory of the current device, 16-byte aligned.
hmc_status check_dev_ptr(hmc_handle *h, const void *p, const char *what) {
    if (!p) return fail(h, HMC_ERR_ARG, std::string("NULL ") + what);
    if (reinterpret_cast<uintptr_t>(p) & 15) return fail(h, HMC_ERR_ARG, std::string(what) + " must be 16-byte aligned");
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, HMC_ERR_ARG, std::string(what) + " is not a CUDA pointer");
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(h, HMC_ERR_CUDA, "cudaGetDevice");
    if (!((at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev))
        return fail(h, HMC_ERR_ARG, std::string(what) + " is not device memory of the current device");
    return HMC_OK;
}
}  // namespace

hmc_status hmc_set_spins_dev(hmc_handle *h, const uint16_t *d_spins) {
    if (h) ++h->state_version;
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if ((s = check_dev_ptr(h, d_spins, "device spins")) != HMC_OK) return s;
    const RepHost &R = selr(h);
    int bad = 0;
    HMC_CK(h, cudaMemsetAsync(&sel_st(h)->bad_spin, 0, sizeof(int32_t), h->stream), "memset");
    HMC_CK(h, hmc::launch_check_spins(d_spins, R.N, h->p.n_orient, sel_st(h), h->stream), "spin check");
    HMC_CK(h, cudaMemcpyAsync(&bad, &sel_st(h)->bad_spin, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream),
           "download");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    if (bad) return fail(h, HMC_ERR_ARG, "spin value >= n_orient");
    HMC_CK(h, hmc::launch_pack_spins(d_spins, h->spins + R.blk_off, R.p.nx, R.p.ny, R.p.nz, h->stream),
           "pack spins");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    return HMC_OK;
}

hmc_status hmc_get_spins_dev(hmc_handle *h, uint16_t *d_spins) {
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if ((s = check_dev_ptr(h, d_spins, "device spins")) != HMC_OK) return s;
    const RepHost &R = selr(h);
    HMC_CK(h, hmc::launch_unpack_spins(h->spins + R.blk_off, d_spins, R.p.nx, R.p.ny, R.p.nz, h->stream),
           "unpack spins");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    return HMC_OK;
}

hmc_status hmc_set_orientations_dev(hmc_handle *h, const double *euler, const uint16_t *d_spins) {
    if (!h) return HMC_ERR_ARG;
    hmc_status s = check_dev_ptr(h, d_spins, "device spins");
    if (s != HMC_OK) return s;
    std::vector<uint16_t> host((size_t)h->N_total);
    HMC_CK(h, cudaMemcpy(host.data(), d_spins, sizeof(uint16_t) * host.size(), cudaMemcpyDeviceToHost),
           "spin download");
    return hmc_set_orientations(h, euler, host.data());
}

hmc_status hmc_get_spins(hmc_handle *h, uint16_t *spins) {
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if (!spins) return fail(h, HMC_ERR_ARG, "NULL spins");
    const RepHost &R = selr(h);
    HMC_CK(h, hmc::launch_unpack_spins(h->spins + R.blk_off, h->stage16, R.p.nx, R.p.ny, R.p.nz, h->stream),
           "unpack spins");
    HMC_CK(h, cudaMemcpyAsync(spins, h->stage16, sizeof(uint16_t) * R.N, cudaMemcpyDeviceToHost, h->stream),
           "spin download");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    return HMC_OK;
}

hmc_status hmc_compute_stress(hmc_handle *h, double *mean, double *energy) {
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if (fault("nan")) {
        HMC_CK(h, cudaMemsetAsync(static_cast<char *>(h->u[h->cur]) + h->tsize * 3 * (size_t)selr(h).blk_off, 0xff,
                                  h->tsize, h->stream),
               "fault injection");
        ++h->state_version;
    }
    HMC_CK(h, enq_stress(h, true, h->stream), "stress launch");
    HMC_CK(h, hmc::launch_end_mcs(h->d_reps, h->R, h->partials, h->nctas, 0, 0, h->stream), "reduction launch");
    if (mean || energy) return read_stats(h, mean, energy);
    return HMC_OK;
}

hmc_status hmc_mpm_steps(hmc_handle *h, int32_t nsteps, double *energy) {
    if (h) ++h->state_version;
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if (nsteps < 0) return fail(h, HMC_ERR_ARG, "nsteps < 0");
    if (fault("launch")) return fail(h, HMC_ERR_CUDA, "injected launch failure (HMC_FAULT=launch)");
    if (nsteps > 0 && (s = ensure_tuned(h)) != HMC_OK) return s;
    for (int k = 0; k < nsteps; ++k) HMC_CK(h, enq_mpm(h, h->stream), "MPM launch");
    if (energy) return hmc_compute_stress(h, nullptr, energy);
    return HMC_OK;
}

hmc_status hmc_sweep_half(hmc_handle *h, int32_t colour, int64_t *accepted) {
    if (h) ++h->state_version;
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if (colour != 0 && colour != 1) return fail(h, HMC_ERR_ARG, "colour must be 0 or 1");
    HMC_CK(h, reset_accepted(h), "memset");
    HMC_CK(h, enq_sweep(h, colour, h->stream), "sweep launch");
    if (fault("copy_lost")) {
        // fault injection on the host: record what a CTA records when its stress copy never
        // lands (wait_timeout = 2), so that the reporting path runs without any GPU fault
        static const int32_t lost = 2;
        HMC_CK(h, cudaMemcpyAsync(&sel_st(h)->wait_timeout, &lost, sizeof(lost), cudaMemcpyHostToDevice, h->stream),
               "fault injection");
        HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    }
    if (accepted) return read_accepted(h, accepted);
    return HMC_OK;
}

hmc_status hmc_sweep_half_margins(hmc_handle *h, int32_t colour, double *margin, int64_t *accepted) {
    if (h) ++h->state_version;
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if (colour != 0 && colour != 1) return fail(h, HMC_ERR_ARG, "colour must be 0 or 1");
    if (!margin) return fail(h, HMC_ERR_ARG, "NULL margin");
    if (h->R != 1) return fail(h, HMC_ERR_ARG, "hmc_sweep_half_margins takes a single-replica handle");
    if (!sweeps_read_stress(h))
        return fail(h, HMC_ERR_ARG, "hmc_sweep_half_margins needs a point-zone elastic term and store_stress = 1");
    const size_t bytes = sizeof(double) * (size_t)h->N_total;
    double *d = nullptr;
    HMC_CK(h, cudaMalloc(&d, bytes), "margin buffer");
    cudaError_t e = cudaMemsetAsync(d, 0xff, bytes, h->stream);   // all-ones words: NaN
    if (e == cudaSuccess) e = reset_accepted(h);
    if (e == cudaSuccess) {
        const int mode = h->p.elastic == HMC_ELASTIC_STRAIN ? hmc::SWEEP_STRAIN : hmc::SWEEP_POINT;
        if (h->p.precision == HMC_FP32) {
            hmc::SweepArgs<float> a = sweep_args<float>(h);
            a.margin = d;
            e = hmc::launch_sweep_margin<float>(a, colour, mode, h->stream);
        } else {
            hmc::SweepArgs<double> a = sweep_args<double>(h);
            a.margin = d;
            e = hmc::launch_sweep_margin<double>(a, colour, mode, h->stream);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(margin, d, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(h, e, "margin sweep");
    int64_t acc = 0;
    if ((s = read_accepted(h, &acc)) != HMC_OK) return s;
    if (accepted) *accepted = acc;
    return HMC_OK;
}

hmc_status hmc_mpm_steps_plain(hmc_handle *h, int32_t nsteps) {
    if (h) ++h->state_version;
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if (nsteps < 0) return fail(h, HMC_ERR_ARG, "nsteps < 0");
    if (h->R != 1 || h->p.precision != HMC_FP64)
        return fail(h, HMC_ERR_ARG, "hmc_mpm_steps_plain takes a single-replica FP64 handle");
    const RepHost &R = h->reps[0];
    if (!h->plain_sig) {
        HMC_CK(h, cudaMalloc(&h->plain_sig, sizeof(double) * 48 * (size_t)R.nblk), "plain step stresses");
        if (cudaMalloc(&h->plain_f, sizeof(double) * 24 * (size_t)R.nblk) != cudaSuccess) {
            cudaFree(h->plain_sig);
            h->plain_sig = nullptr;
            return fail(h, HMC_ERR_OOM, "plain step cell forces");
        }
    }
    hmc::PlainArgs a;
    a.spins = h->spins;
    a.ctab = static_cast<const double *>(h->ctab);
    a.st = h->st;
    a.v = static_cast<double *>(h->v);
    a.sig = h->plain_sig;
    a.fcell = h->plain_f;
    a.dt = h->dt;
    a.dt_over_m = h->dt / 8.0;   // lumped mass rho * V * sum_p N_I(x_p) = 8 voxels
    a.keep = 1.0 - h->damping;
    a.nbx = R.nbx;
    a.nby = R.nby;
    a.nbz = R.nbz;
    a.nblk = (int)R.nblk;
    a.u = static_cast<const double *>(h->u[h->cur]);
    a.u_out = nullptr;
    HMC_CK(h, hmc::launch_plain_init(a, h->stream), "plain step stress");
    for (int k = 0; k < nsteps; ++k) {
        a.u = static_cast<const double *>(h->u[h->cur]);
        a.u_out = static_cast<double *>(h->u[h->cur ^ 1]);
        HMC_CK(h, hmc::launch_plain_step(a, h->stream), "plain step");
        h->cur ^= 1;
    }
    return HMC_OK;
}

hmc_status hmc_end_mcs(hmc_handle *h) {
    if (h) ++h->state_version;
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    HMC_CK(h, hmc::launch_end_mcs(h->d_reps, h->R, h->partials, h->nctas, 1, 1, h->stream), "end-of-step launch");
    return HMC_OK;
}

hmc_status hmc_mc_sweeps(hmc_handle *h, int32_t n_mcs, int64_t *accepted) {
    if (h) ++h->state_version;
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if (n_mcs < 0) return fail(h, HMC_ERR_ARG, "n_mcs < 0");
    if (fault("launch")) return fail(h, HMC_ERR_CUDA, "injected launch failure (HMC_FAULT=launch)");
    if (n_mcs > 0 && h->p.mpm_steps_per_mcs > 0 && (s = ensure_tuned(h)) != HMC_OK) return s;
    HMC_CK(h, reset_accepted(h), "memset");
    for (int m = 0; m < n_mcs; ++m) {
        const int c0 = h->cur;
        if (!h->gexec[c0]) {
            // capture one step of every replica starting from this displacement buffer
            cudaGraph_t g = nullptr;
            HMC_CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
            cudaError_t e = enqueue_mcs(h, h->cap);
            cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
            h->cur = c0;
            if (e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return cuda_fail(h, e, "capture");
            }
            if (e2 != cudaSuccess) return cuda_fail(h, e2, "end capture");
            e = cudaGraphInstantiate(&h->gexec[c0], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                h->gexec[c0] = nullptr;
                return cuda_fail(h, e, "graph instantiate");
            }
        }
        HMC_CK(h, cudaGraphLaunch(h->gexec[c0], h->stream), "graph launch");
        if (h->p.mpm_steps_per_mcs & 1) h->cur ^= 1;
    }
    if (accepted) return read_accepted(h, accepted);
    return HMC_OK;
}

hmc_status hmc_grain_count(hmc_handle *h, int64_t *n_grains) {
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if (!n_grains) return fail(h, HMC_ERR_ARG, "NULL n_grains");
    const RepHost &R = selr(h);
    if (R.N > 0xffffffffll) return fail(h, HMC_ERR_ARG, "replica too large for 32-bit grain labels");
    if (!h->cc_parent) HMC_CK(h, cudaMalloc(&h->cc_parent, sizeof(unsigned) * (size_t)h->N_max), "grain labels");
    if (!h->cc_count) HMC_CK(h, cudaMalloc(&h->cc_count, 2 * sizeof(unsigned long long)), "grain count");
    int *err = reinterpret_cast<int *>(h->cc_count + 1);
    HMC_CK(h, hmc::launch_grain_count(h->spins + R.blk_off, R.nbx, R.nby, R.nbz, h->cc_parent, h->cc_count, err,
                                      h->stream),
           "grain count launch");
    unsigned long long host[2] = {0, 0};
    HMC_CK(h, cudaMemcpyAsync(host, h->cc_count, sizeof(host), cudaMemcpyDeviceToHost, h->stream), "grain count read");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    if ((int)(host[1] & 0xffffffffu) != 0) return fail(h, HMC_ERR_TIMEOUT, "grain union-find exceeded its iteration cap");
    *n_grains = (int64_t)host[0];
    return HMC_OK;
}

hmc_status hmc_texture_histogram(hmc_handle *h, int32_t kind, int32_t nbins, double *fractions,
                                 int64_t *counts_per_q) {
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    const int Q = h->p.n_orient;
    const RepHost &R = selr(h);
    if (fractions) {
        if (kind == HMC_HIST_PER_Q && nbins != Q) return fail(h, HMC_ERR_ARG, "PER_Q needs nbins == n_orient");
        if (kind != HMC_HIST_PER_Q && kind != HMC_HIST_ANGLE_100 && kind != HMC_HIST_YOUNG)
            return fail(h, HMC_ERR_ARG, "bad kind");
        if (nbins < 1) return fail(h, HMC_ERR_ARG, "nbins < 1");
    }
    HMC_CK(h, cudaMemsetAsync(h->counts, 0, sizeof(unsigned long long) * Q, h->stream), "memset");
    HMC_CK(h, cudaMemsetAsync(&sel_st(h)->unlike, 0, sizeof(unsigned long long), h->stream), "memset");
    HMC_CK(h, hmc::launch_bonds_counts(h->spins + R.blk_off, R.nbx, R.nby, R.nbz, Q, h->counts, sel_st(h), h->stream),
           "counts launch");
    if (fractions) {
        std::vector<int32_t> map(Q);
        for (int q = 0; q < Q; ++q) {
            const double *A = &h->A[(size_t)q * 9];
            int b = q;
            if (kind == HMC_HIST_ANGLE_100) {
                double c = 0;
                for (int m = 0; m < 3; ++m) {
                    const double d =
                        std::fabs(A[0 * 3 + m] * R.axis[0] + A[1 * 3 + m] * R.axis[1] + A[2 * 3 + m] * R.axis[2]);
                    c = std::fmax(c, d);
                }
                const double ang = std::acos(std::fmin(1.0, c)) * 180.0 / M_PI;
                b = (int)(ang / (90.0 / nbins));
            } else if (kind == HMC_HIST_YOUNG) {
                double N[6], Nsv[6];
                axis_vectors(R.axis, N, Nsv);
                double nsn = 0;
                for (int i = 0; i < 6; ++i)
                    for (int j = 0; j < 6; ++j) nsn += N[i] * h->Sv[(size_t)q * 36 + 6 * i + j] * N[j];
                const double x = 1.0 / nsn / h->p.c11;
                const double sd = h->S11 - h->S12 - 0.5 * h->S44;
                const double e1 = 1.0 / h->S11 / h->p.c11, e2 = 1.0 / (h->S11 - 2.0 * sd / 3.0) / h->p.c11;
                const double lo = std::fmin(e1, e2), hi = std::fmax(e1, e2);
                b = hi > lo ? (int)((x - lo) / (hi - lo) * nbins) : 0;
            }
            map[q] = b < 0 ? 0 : (b >= nbins ? nbins - 1 : b);
        }
        if (h->bins_cap < nbins) {
            HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
            if (h->bins) cudaFree(h->bins);
            if (h->fractions) cudaFree(h->fractions);
            h->bins = nullptr;
            h->fractions = nullptr;
            h->bins_cap = 0;
            HMC_CK(h, cudaMalloc(&h->bins, sizeof(unsigned long long) * nbins), "bins");
            HMC_CK(h, cudaMalloc(&h->fractions, sizeof(double) * nbins), "fractions");
            h->bins_cap = nbins;
        }
        if (!h->binmap) HMC_CK(h, cudaMalloc(&h->binmap, sizeof(int32_t) * Q), "binmap");
        HMC_CK(h, cudaMemcpyAsync(h->binmap, map.data(), sizeof(int32_t) * Q, cudaMemcpyHostToDevice, h->stream),
               "binmap");
        HMC_CK(h, cudaMemsetAsync(h->bins, 0, sizeof(unsigned long long) * nbins, h->stream), "memset");
        HMC_CK(h, hmc::launch_bins(h->counts, h->binmap, Q, nbins, h->bins, h->fractions, R.N, h->stream),
               "bins launch");
        HMC_CK(h, cudaMemcpyAsync(fractions, h->fractions, sizeof(double) * nbins, cudaMemcpyDeviceToHost, h->stream),
               "download");
    }
    if (counts_per_q)
        HMC_CK(h, cudaMemcpyAsync(counts_per_q, h->counts, sizeof(int64_t) * Q, cudaMemcpyDeviceToHost, h->stream),
               "download");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    return HMC_OK;
}

hmc_status hmc_energy(hmc_handle *h, int64_t *unlike, double *energy, double *mean) {
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    const RepHost &R = selr(h);
    if (unlike) {
        HMC_CK(h, cudaMemsetAsync(h->counts, 0, sizeof(unsigned long long) * h->p.n_orient, h->stream), "memset");
        HMC_CK(h, cudaMemsetAsync(&sel_st(h)->unlike, 0, sizeof(unsigned long long), h->stream), "memset");
        HMC_CK(h, hmc::launch_bonds_counts(h->spins + R.blk_off, R.nbx, R.nby, R.nbz, h->p.n_orient, h->counts,
                                           sel_st(h), h->stream),
               "bonds launch");
        unsigned long long u = 0;
        HMC_CK(h, cudaMemcpyAsync(&u, &sel_st(h)->unlike, sizeof(u), cudaMemcpyDeviceToHost, h->stream), "download");
        HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
        *unlike = (int64_t)u;
    }
    if (energy || mean) return read_stats(h, mean, energy);
    return HMC_OK;
}

hmc_status hmc_get_stress(hmc_handle *h, double *sigma) {
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if (!sigma) return fail(h, HMC_ERR_ARG, "NULL sigma");
    const RepHost &R = selr(h);
    const size_t n = 48 * (size_t)R.nblk;
    const char *src = static_cast<const char *>(h->sig) + h->tsize * 48 * (size_t)R.blk_off;
    if (h->p.precision == HMC_FP32) {
        std::vector<float> t(n);
        HMC_CK(h, cudaMemcpyAsync(t.data(), src, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream), "download");
        HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
        unpack_stress_host<float>(R, t, sigma);
    } else {
        std::vector<double> t(n);
        HMC_CK(h, cudaMemcpyAsync(t.data(), src, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "download");
        HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
        unpack_stress_host<double>(R, t, sigma);
    }
    return HMC_OK;
}

hmc_status hmc_set_stress(hmc_handle *h, const double *sigma) {
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if (!sigma) return fail(h, HMC_ERR_ARG, "NULL sigma");
    const RepHost &R = selr(h);
    for (long long i = 0; i < 6 * R.N; ++i)
        if (!std::isfinite(sigma[i])) return fail(h, HMC_ERR_ARG, "non-finite stress");
    const size_t n = 48 * (size_t)R.nblk;
    char *dst = static_cast<char *>(h->sig) + h->tsize * 48 * (size_t)R.blk_off;
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    if (h->p.precision == HMC_FP32) {
        std::vector<float> t(n);
        pack_stress_host<float>(R, sigma, t);
        HMC_CK(h, cudaMemcpy(dst, t.data(), n * sizeof(float), cudaMemcpyHostToDevice), "upload");
    } else {
        std::vector<double> t(n);
        pack_stress_host<double>(R, sigma, t);
        HMC_CK(h, cudaMemcpy(dst, t.data(), n * sizeof(double), cudaMemcpyHostToDevice), "upload");
    }
    return HMC_OK;
}

hmc_status hmc_get_nodal(hmc_handle *h, double *u, double *v) {
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if (u && (s = nodal_io(h, h->u[h->cur], u, true)) != HMC_OK) return s;
    if (v && (s = nodal_io(h, h->v, v, true)) != HMC_OK) return s;
    return HMC_OK;
}

hmc_status hmc_set_nodal(hmc_handle *h, const double *u, const double *v) {
    if (h) ++h->state_version;
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    const size_t n = 3 * (size_t)selr(h).nblk;
    for (const double *a : {u, v})
        if (a)
            for (size_t i = 0; i < n; ++i)
                if (!std::isfinite(a[i])) return fail(h, HMC_ERR_ARG, "non-finite nodal value");
    if (u && (s = nodal_io(h, h->u[h->cur], const_cast<double *>(u), false)) != HMC_OK) return s;
    if (v && (s = nodal_io(h, h->v, const_cast<double *>(v), false)) != HMC_OK) return s;
    // a finite nodal state clears the replica's non-finite flag
    HMC_CK(h, cudaMemsetAsync(&sel_st(h)->nonfinite, 0, sizeof(int32_t), h->stream), "memset");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    return HMC_OK;
}

hmc_status hmc_get_strain(hmc_handle *h, double *e) {
    if (!h) return HMC_ERR_ARG;
    if (!e) return fail(h, HMC_ERR_ARG, "NULL strain");
    HMC_CK(h, cudaMemcpyAsync(e, sel_st(h)->ebar, sizeof(double) * 6, cudaMemcpyDeviceToHost, h->stream), "download");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    return HMC_OK;
}

hmc_status hmc_set_strain(hmc_handle *h, const double *e) {
    if (h) ++h->state_version;
    if (!h) return HMC_ERR_ARG;
    if (!e) return fail(h, HMC_ERR_ARG, "NULL strain");
    double d[6];
    float f[6];
    for (int i = 0; i < 6; ++i) {
        if (!std::isfinite(e[i])) return fail(h, HMC_ERR_ARG, "non-finite strain");
        d[i] = e[i];
        f[i] = (float)e[i];
    }
    HMC_CK(h, cudaMemcpyAsync(sel_st(h)->ebar, d, sizeof(d), cudaMemcpyHostToDevice, h->stream), "upload");
    HMC_CK(h, cudaMemcpyAsync(sel_st(h)->ebar_f, f, sizeof(f), cudaMemcpyHostToDevice, h->stream), "upload");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    return HMC_OK;
}

hmc_status hmc_set_load(hmc_handle *h, double value) {
    if (h) ++h->state_version;
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if (!std::isfinite(value)) return fail(h, HMC_ERR_ARG, "non-finite load");
    const int bc = selr(h).p.bc;
    if (bc != HMC_BC_UNIAXIAL && bc != HMC_BC_TRACTION) return fail(h, HMC_ERR_ARG, "STRAIN6 has no scalar load");
    DevState st;
    HMC_CK(h, cudaMemcpyAsync(&st, sel_st(h), sizeof(st), cudaMemcpyDeviceToHost, h->stream), "download");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    if (bc == HMC_BC_UNIAXIAL) {
        for (int i = 0; i < 6; ++i) st.ebar[i] += (value - st.eps0) / st.axNB * st.axB[i];
        st.eps0 = value;
    } else {
        double e[6];
        for (int i = 0; i < 6; ++i) {
            double d = 0;
            for (int j = 0; j < 6; ++j) d += st.sr[6 * i + j] * (value - st.sig0) * st.axN[j];
            e[i] = st.ebar[i] + d;
        }
        for (int i = 0; i < 6; ++i) st.ebar[i] = e[i];
        st.sig0 = value;
    }
    for (int i = 0; i < 6; ++i) st.ebar_f[i] = (float)st.ebar[i];
    DevState *d = sel_st(h);
    HMC_CK(h, cudaMemcpyAsync(d->ebar, st.ebar, sizeof(st.ebar), cudaMemcpyHostToDevice, h->stream), "upload");
    HMC_CK(h, cudaMemcpyAsync(d->ebar_f, st.ebar_f, sizeof(st.ebar_f), cudaMemcpyHostToDevice, h->stream), "upload");
    HMC_CK(h, cudaMemcpyAsync(&d->eps0, &st.eps0, sizeof(double), cudaMemcpyHostToDevice, h->stream), "upload");
    HMC_CK(h, cudaMemcpyAsync(&d->sig0, &st.sig0, sizeof(double), cudaMemcpyHostToDevice, h->stream), "upload");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    return HMC_OK;
}

hmc_status hmc_get_info(hmc_handle *h, hmc_info *info) {
    if (!h) return HMC_ERR_ARG;
    if (!info) return fail(h, HMC_ERR_ARG, "NULL info");
    DevState st;
    HMC_CK(h, cudaMemcpyAsync(&st, sel_st(h), sizeof(st), cudaMemcpyDeviceToHost, h->stream), "download");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    const RepHost &R = selr(h);
    info->dt = h->dt;
    info->damping = h->damping;
    info->elastic_scale = R.lam;
    for (int i = 0; i < 6; ++i) info->strain_bar[i] = st.ebar[i];
    info->mcs = st.mcs;
    info->u_buffer = h->cur;
    info->n_sites = R.N;
    info->n_nodes = R.nblk;
    info->zone_trials = 0;
    if (h->zone_count) {
        unsigned n = 0;
        HMC_CK(h, cudaMemcpy(&n, h->zone_count, sizeof(n), cudaMemcpyDeviceToHost), "download");
        info->zone_trials = n;
    }
    return HMC_OK;
}

hmc_status hmc_get_state(hmc_handle *h, void *buf, size_t *bytes) {
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if (!bytes) return fail(h, HMC_ERR_ARG, "NULL bytes");
    const RepHost &R = selr(h);
    const size_t need = sizeof(StateHeader) + 2 * (size_t)R.N + 2 * 3 * 8 * (size_t)R.nblk;
    if (!buf) {
        *bytes = need;
        return HMC_OK;
    }
    if (*bytes < need) return fail(h, HMC_ERR_ARG, "buffer too small");
    StateHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, "HMCSTAT1", 8);
    hd.nx = R.p.nx; hd.ny = R.p.ny; hd.nz = R.p.nz; hd.precision = h->p.precision;
    DevState st;
    HMC_CK(h, cudaMemcpyAsync(&st, sel_st(h), sizeof(st), cudaMemcpyDeviceToHost, h->stream), "download");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    hd.mcs = st.mcs;
    for (int i = 0; i < 6; ++i) hd.ebar[i] = st.ebar[i];
    char *p = static_cast<char *>(buf);
    std::memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    if ((s = hmc_get_spins(h, reinterpret_cast<uint16_t *>(p))) != HMC_OK) return s;
    p += 2 * (size_t)R.N;
    double *u = reinterpret_cast<double *>(p), *v = u + 3 * (size_t)R.nblk;
    if ((s = hmc_get_nodal(h, u, v)) != HMC_OK) return s;
    *bytes = need;
    return HMC_OK;
}

hmc_status hmc_set_state(hmc_handle *h, const void *buf, size_t bytes) {
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    const RepHost &R = selr(h);
    const size_t need = sizeof(StateHeader) + 2 * (size_t)R.N + 2 * 3 * 8 * (size_t)R.nblk;
    if (!buf || bytes < need) return fail(h, HMC_ERR_ARG, "state buffer too small");
    StateHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    if (std::memcmp(hd.magic, "HMCSTAT1", 8) != 0 || hd.nx != R.p.nx || hd.ny != R.p.ny || hd.nz != R.p.nz)
        return fail(h, HMC_ERR_ARG, "state does not match this replica");
    const char *p = static_cast<const char *>(buf) + sizeof(hd);
    if ((s = hmc_set_spins(h, reinterpret_cast<const uint16_t *>(p))) != HMC_OK) return s;
    p += 2 * (size_t)R.N;
    const double *u = reinterpret_cast<const double *>(p), *v = u + 3 * (size_t)R.nblk;
    if ((s = hmc_set_nodal(h, u, v)) != HMC_OK) return s;
    if ((s = hmc_set_strain(h, hd.ebar)) != HMC_OK) return s;
    HMC_CK(h, cudaMemcpyAsync(&sel_st(h)->mcs, &hd.mcs, sizeof(uint32_t), cudaMemcpyHostToDevice, h->stream),
           "upload");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    return HMC_OK;
}

hmc_status hmc_synchronize(hmc_handle *h) {
    if (!h) return HMC_ERR_ARG;
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    return HMC_OK;
}

const char *hmc_last_error(const hmc_handle *h) { return h ? h->err.c_str() : g_create_error.c_str(); }

}  // extern "C"

// ---- adjoint of the explicit MPM solve ---------------------------------------

namespace {

template <typename T>
cudaError_t mpm_custom(hmc_handle *h, const void *uin, void *uout, void *v, const hmc::Replica *reps, double keep) {
    hmc::MpmArgs<T> a = mpm_args<T>(h, uin, uout, v);
    a.reps = reps;
    a.keep = (T)keep;
    return hmc::launch_mpm_step<T>(a, h->mpm_shape, h->stream);
}


template <typename T>
hmc::AdjArgs<T> adj_args(hmc_handle *h) {
    hmc::AdjArgs<T> a;
    const RepHost &R = h->reps[0];
    a.spins = h->spins;
    a.ctab = static_cast<const T *>(h->ctab);
    a.rtab = static_cast<const T *>(h->adj.rtab);
    a.wtab = static_cast<const T *>(h->wtab);
    a.partials = h->adj.partials;
    for (int i = 0; i < 6; ++i) a.ebar[i] = (T)h->adj.ebar[i];
    a.nx = R.p.nx; a.ny = R.p.ny; a.nz = R.p.nz;
    a.nbx = R.nbx; a.nby = R.nby; a.nbz = R.nbz;
    a.nblk = (int)R.nblk;
    return a;
}

char *seg_ptr(hmc_handle *h, void *base, int j) { return static_cast<char *>(base) + (size_t)j * node_bytes(h); }

hmc_status adj_alloc(hmc_handle *h, int steps, int ck) {
    auto &A = h->adj;
    const int nseg = (steps + ck - 1) / ck;
    if (A.lam && A.steps == steps && A.ck == ck) return HMC_OK;
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    free_adjoint(h);
    const RepHost &R = h->reps[0];
    const size_t nb = node_bytes(h);
    A.nctas = (int)((R.nblk + 255) / 256);
    struct Alloc { void **ptr; size_t bytes; const char *what; };
    Alloc allocs[] = {
        {&A.rtab, h->tsize * 72 * (size_t)h->p.n_orient, "basis tables"},
        {&A.lam, nb, "adjoint lambda"}, {&A.ubar, nb, "adjoint u"}, {&A.tmp, nb, "adjoint scratch"},
        {&A.vtmp, nb, "segment velocity"}, {&A.seg, nb * (size_t)ck, "segment states"},
        {&A.ck_u, nb * (size_t)nseg, "checkpoints u"}, {&A.ck_v, nb * (size_t)nseg, "checkpoints v"},
        {&A.w, h->tsize * (size_t)R.N, "field w"}, {&A.g, h->tsize * (size_t)R.N, "cotangent field"},
        {&A.fcell, h->tsize * 24 * (size_t)R.nblk, "cell contributions"},
        {(void **)&A.partials, sizeof(double) * 10 * (size_t)A.nctas, "adjoint partials"},
        {(void **)&A.grad, sizeof(double) * 10, "gradient"},
        {(void **)&A.reps0, sizeof(hmc::Replica), "adjoint descriptor"},
        {(void **)&A.st0, sizeof(DevState), "adjoint state"},
    };
    for (auto &a : allocs) {
        cudaError_t e = cudaMalloc(a.ptr, a.bytes);
        if (e != cudaSuccess) {
            free_adjoint(h);
            return cuda_fail(h, e, a.what);
        }
    }
    A.steps = steps;
    A.ck = ck;
    A.nseg = nseg;
    // the replica's descriptor with a zero mean strain, for F(lambda; Ebar = 0)
    hmc::Replica rd;
    HMC_CK(h, cudaMemcpy(&rd, h->d_reps, sizeof(rd), cudaMemcpyDeviceToHost), "descriptor download");
    rd.st = A.st0;
    DevState z;
    std::memset(&z, 0, sizeof(z));
    HMC_CK(h, cudaMemcpy(A.reps0, &rd, sizeof(rd), cudaMemcpyHostToDevice), "descriptor upload");
    HMC_CK(h, cudaMemcpy(A.st0, &z, sizeof(z), cudaMemcpyHostToDevice), "state upload");
    return HMC_OK;
}

// Rotated basis tensors R_1, R_2, R_3 (C' = C11 R_1 + C12 R_2 + C44 R_3) by the
// same Bond transform as the stiffness table.
hmc_status adj_tables(hmc_handle *h) {
    auto &A = h->adj;
    if (A.rtab_version == h->orient_version) return HMC_OK;
    const int Q = h->p.n_orient;
    std::vector<double> Rv((size_t)Q * 3 * 36);
    for (int i = 0; i < 3; ++i) {
        double B[36] = {0};
        const double c11 = i == 0, c12 = i == 1, c44 = i == 2;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) B[6 * a + b] = (a == b) ? c11 : c12;
        for (int a = 3; a < 6; ++a) B[6 * a + a] = c44;
        for (int q = 0; q < Q; ++q) {
            double M[36], Ns[36];
            bond(&h->A[(size_t)q * 9], M, Ns);
            congruence(M, B, &Rv[((size_t)q * 3 + i) * 36]);
        }
    }
    auto pack = [&](auto tag) -> hmc_status {
        using T = decltype(tag);
        std::vector<T> out((size_t)Q * 72, T(0));
        for (int q = 0; q < Q; ++q)
            for (int i = 0; i < 3; ++i) {
                int n = 0;
                for (int a = 0; a < 6; ++a)
                    for (int b = a; b < 6; ++b) out[(size_t)q * 72 + 24 * i + n++] = (T)Rv[((size_t)q * 3 + i) * 36 + 6 * a + b];
            }
        HMC_CK(h, cudaMemcpy(A.rtab, out.data(), out.size() * sizeof(T), cudaMemcpyHostToDevice), "basis upload");
        return HMC_OK;
    };
    hmc_status s = h->p.precision == HMC_FP32 ? pack(float()) : pack(double());
    if (s != HMC_OK) return s;
    A.rtab_version = h->orient_version;
    return HMC_OK;
}

template <typename T>
cudaError_t adj_terminal(hmc_handle *h, const T *g, double gW, T *w) {
    return hmc::launch_adj_terminal<T>(adj_args<T>(h), static_cast<const T *>(h->u[h->cur]), g, (T)gW, w,
                                       static_cast<T *>(h->adj.fcell), h->stream);
}

template <typename T>
hmc_status adj_backward_t(hmc_handle *h, double gW, const double *g_field, double *grad) {
    auto &A = h->adj;
    const RepHost &R = h->reps[0];
    const double c = h->dt / 8.0;
    const T *g = nullptr;
    if (g_field) {
        std::vector<T> t((size_t)R.N);
        for (long long i = 0; i < R.N; ++i) {
            if (!std::isfinite(g_field[i])) return fail(h, HMC_ERR_ARG, "non-finite cotangent");
            t[i] = (T)g_field[i];
        }
        HMC_CK(h, cudaMemcpyAsync(A.g, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream), "upload");
        HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
        g = static_cast<const T *>(A.g);
    }
    HMC_CK(h, cudaMemsetAsync(A.grad, 0, sizeof(double) * 10, h->stream), "memset");
    // terminal: direct parameter terms and ubar^T = sum_p alpha_p B_p^T sigma_p, lambda^T = dt ubar^T
    HMC_CK(h, adj_terminal<T>(h, g, gW, nullptr), "terminal launch");
    HMC_CK(h, hmc::launch_adj_reduce(A.partials, A.nctas, 10, 10, 1.0, A.grad, h->stream), "reduce launch");
    const hmc::AdjArgs<T> aa = adj_args<T>(h);
    HMC_CK(h, hmc::launch_adj_gather<T>(aa, static_cast<const T *>(A.fcell), T(1), static_cast<T *>(A.ubar), h->stream),
           "gather launch");
    HMC_CK(h, hmc::launch_adj_gather<T>(aa, static_cast<const T *>(A.fcell), (T)h->dt, static_cast<T *>(A.lam),
                                        h->stream),
           "gather launch");
    const size_t nb = node_bytes(h);
    // every reverse step adds its parameter terms to its CTA's partials; one reduction at the end
    HMC_CK(h, cudaMemsetAsync(A.partials, 0, sizeof(double) * 9 * (size_t)A.nctas, h->stream), "memset");
    for (int s = A.nseg - 1; s >= 0; --s) {
        const int n0 = s * A.ck, len = std::min(A.ck, A.steps - n0);
        // recompute the segment's forward states u^{n0} .. u^{n0+len-1} from its checkpoint
        HMC_CK(h, cudaMemcpyAsync(seg_ptr(h, A.seg, 0), seg_ptr(h, A.ck_u, s), nb, cudaMemcpyDeviceToDevice, h->stream),
               "checkpoint copy");
        HMC_CK(h, cudaMemcpyAsync(A.vtmp, seg_ptr(h, A.ck_v, s), nb, cudaMemcpyDeviceToDevice, h->stream),
               "checkpoint copy");
        for (int j = 1; j < len; ++j)
            HMC_CK(h, mpm_custom<T>(h, seg_ptr(h, A.seg, j - 1), seg_ptr(h, A.seg, j), A.vtmp, h->d_reps,
                                    1.0 - h->damping),
                   "recompute launch");
        for (int j = len - 1; j >= 0; --j) {
            HMC_CK(h, hmc::launch_adj_params<T>(aa, static_cast<const T *>(A.lam),
                                                reinterpret_cast<const T *>(seg_ptr(h, A.seg, j)), h->stream),
                   "parameter launch");
            // ubar^n = ubar^{n+1} + c F(lambda^{n+1}; 0); tmp = lambda^{n+1} + dt ubar^n
            HMC_CK(h, mpm_custom<T>(h, A.lam, A.tmp, A.ubar, A.reps0, 1.0), "adjoint step launch");
            HMC_CK(h, hmc::launch_adj_lambda<T>(3ll * R.nblk, static_cast<const T *>(A.tmp), (T)h->damping,
                                                static_cast<T *>(A.lam), h->stream),
                   "lambda launch");
        }
    }
    HMC_CK(h, hmc::launch_adj_reduce(A.partials, A.nctas, 9, 9, -c, A.grad + 1, h->stream), "reduce launch");
    double out[10];
    HMC_CK(h, cudaMemcpyAsync(out, A.grad, sizeof(out), cudaMemcpyDeviceToHost, h->stream), "download");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    for (int k = 0; k < 9; ++k) {
        if (!std::isfinite(out[1 + k])) return fail(h, HMC_ERR_NONFINITE, "non-finite gradient");
        grad[k] = out[1 + k];
    }
    return HMC_OK;
}

}  // namespace

extern "C" {

hmc_status hmc_adjoint_forward(hmc_handle *h, int32_t nsteps, int32_t checkpoint_every, double *W, double *w_field) {
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if (h->R != 1) return fail(h, HMC_ERR_STATE, "the adjoint runs on single-replica handles");
    if (nsteps < 1 || checkpoint_every < 1) return fail(h, HMC_ERR_ARG, "nsteps and checkpoint_every must be >= 1");
    if ((s = ensure_tuned(h)) != HMC_OK) return s;
    if ((s = adj_alloc(h, nsteps, checkpoint_every)) != HMC_OK) return s;
    if ((s = adj_tables(h)) != HMC_OK) return s;
    auto &A = h->adj;
    HMC_CK(h, cudaMemcpyAsync(A.ebar, h->st[0].ebar, sizeof(A.ebar), cudaMemcpyDeviceToHost, h->stream), "download");
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    const size_t nb = node_bytes(h);
    for (int sg = 0; sg < A.nseg; ++sg) {
        HMC_CK(h, cudaMemcpyAsync(seg_ptr(h, A.ck_u, sg), h->u[h->cur], nb, cudaMemcpyDeviceToDevice, h->stream),
               "checkpoint");
        HMC_CK(h, cudaMemcpyAsync(seg_ptr(h, A.ck_v, sg), h->v, nb, cudaMemcpyDeviceToDevice, h->stream), "checkpoint");
        const int len = std::min(A.ck, A.steps - sg * A.ck);
        for (int j = 0; j < len; ++j) HMC_CK(h, enq_mpm(h, h->stream), "MPM launch");
    }
    HMC_CK(h, cudaMemsetAsync(A.grad, 0, sizeof(double) * 10, h->stream), "memset");
    if (h->p.precision == HMC_FP32)
        HMC_CK(h, adj_terminal<float>(h, nullptr, 0.0, static_cast<float *>(A.w)), "terminal launch");
    else
        HMC_CK(h, adj_terminal<double>(h, nullptr, 0.0, static_cast<double *>(A.w)), "terminal launch");
    HMC_CK(h, hmc::launch_adj_reduce(A.partials, A.nctas, 10, 10, 1.0, A.grad, h->stream), "reduce launch");
    const RepHost &R = h->reps[0];
    if (W) HMC_CK(h, cudaMemcpyAsync(W, A.grad, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "download");
    if (w_field) {
        if (h->p.precision == HMC_FP32) {
            std::vector<float> t((size_t)R.N);
            HMC_CK(h, cudaMemcpyAsync(t.data(), A.w, t.size() * 4, cudaMemcpyDeviceToHost, h->stream), "download");
            HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
            for (long long i = 0; i < R.N; ++i) w_field[i] = t[i];
        } else {
            HMC_CK(h, cudaMemcpyAsync(w_field, A.w, (size_t)R.N * 8, cudaMemcpyDeviceToHost, h->stream), "download");
        }
    }
    HMC_CK(h, cudaStreamSynchronize(h->stream), "sync");
    ++h->state_version;
    A.state_version = h->state_version;
    A.have_forward = true;
    return HMC_OK;
}

hmc_status hmc_adjoint_backward(hmc_handle *h, double gW, const double *g_field, double *grad) {
    hmc_status s = need_oriented(h);
    if (s != HMC_OK) return s;
    if (!grad) return fail(h, HMC_ERR_ARG, "NULL grad");
    if (!std::isfinite(gW)) return fail(h, HMC_ERR_ARG, "non-finite gW");
    if (!h->adj.have_forward || h->adj.state_version != h->state_version || h->adj.rtab_version != h->orient_version)
        return fail(h, HMC_ERR_STATE, "hmc_adjoint_backward needs the state left by hmc_adjoint_forward");
    return h->p.precision == HMC_FP32 ? adj_backward_t<float>(h, gW, g_field, grad)
                                      : adj_backward_t<double>(h, gW, g_field, grad);
}

}  // extern "C"
