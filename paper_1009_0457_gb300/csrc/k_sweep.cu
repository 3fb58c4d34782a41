// Red/black checkerboard half sweep (Sec. "Microstructural Evolution") with the
// Metropolis rule (Eq. 5) on the bond-energy change of the Potts Hamiltonian
// (Eq. 4, bonds counted once, 6 neighbours, periodic) plus the one-point
// constant-traction zone shift (Eqs. 6-8 and 13) from the stored stress, or its
// constant-strain reading.
//
// One thread per 2x2x2 block: it draws the trials of the block's four sites of
// the sweep's colour; a tile of 256 blocks of one replica is one CTA's work.
// Per block the sweep reads the block's 16 B of spins, the other colour's 8 B
// quad of the six face neighbours and (stored-stress elastic forms) the colour's
// 96 B of stress (FP32), and writes the colour's 8 B quad when a site changed.
// Same-colour sites share no neighbour, so the in-place update is race free.
// The colour's four sites of a block share one Philox4x32-10 block (a word each).
// The bond counts compare the six neighbours as three pairs of 16-bit halves with
// per-half SIMD minima: six minima in place of twelve compares, the same integers.
//
// Five CTAs per SM (FP32).  With the stored stress, thread 0 starts a bulk
// asynchronous copy of the tile's stress of the colour into shared memory
// (completing on an mbarrier) as the CTA begins; the threads meanwhile load their
// spins and neighbours and run the Philox and bond arithmetic.  With an elastic
// term, the trials that change the orientation (a minority: interior sites copy
// their own orientation) are listed in shared memory, each warp in its own region
// (positions from ballots, no shared counter), and only thread 0 waits for the
// copy: one CTA barrier then publishes the staged stress, after which each warp
// evaluates its listed trials densely with its 32 lanes (zone energies and the
// logarithm of the Metropolis threshold on full lanes rather than on the few whose
// site needs them) and its lanes apply their decisions after a warp barrier.  The
// last warp to finish adds the CTA's acceptances to the replica's count.
//
// With the 27-point zone the sweep only lists its non-trivial trials (site,
// replica, old and new orientation, the acceptance draw) in global memory with
// one atomic per warp; the zone kernel decides them.
#include "hmc_device.cuh"

namespace hmc {

namespace {

constexpr unsigned FULL = 0xffffffffu;
// threads (= blocks) of a sweep CTA: a tile of BLOCK_THREADS blocks is one CTA of 256 threads
// or split over two of 128 (a tuning knob of the stored-stress point-zone and pure Potts forms;
// measured on the 256^3 workload: 256 threads 0.073 ms, 128 0.078 ms, 64 0.088 ms per half
// sweep, the per-CTA costs outweighing the shorter barriers).  Decisions do not depend on it.
constexpr int SWEEP_CTA = 256;
template <int CTA>
__host__ __device__ constexpr int split_of() {
    static_assert(BLOCK_THREADS % CTA == 0, "tiles split evenly");
    static_assert(4 * CTA <= 1024, "a trial's thread and slot fit ten bits");
    return BLOCK_THREADS / CTA;
}

// Phi(q; sigma) = sum over the three crystal axes of p_m^2, p_m = a_m . sigma . a_m.
// For one cubic material the zone energy w(q) = 1/2 sigma.S'(q).sigma =
// 1/2 [S12 tr^2 + S44/2 |sigma|^2 + s_d Phi(q)], so
// w(q_old) - w(q_new) = s_d / 2 (Phi(q_old) - Phi(q_new)).  The axes are orthonormal,
// so p_2 = tr sigma - p_0 - p_1 and two axes per orientation suffice (an 8-value
// row, two 16-byte loads).
template <typename T>
struct AxisRow;
template <>
struct AxisRow<float> {
    float v[8];
    __device__ __forceinline__ void load(const float *p) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
        const float4 t0 = __ldg(q), t1 = __ldg(q + 1);
        v[0] = t0.x; v[1] = t0.y; v[2] = t0.z; v[3] = t0.w;
        v[4] = t1.x; v[5] = t1.y; v[6] = t1.z; v[7] = t1.w;
    }
};
template <>
struct AxisRow<double> {
    double v[8];
    __device__ __forceinline__ void load(const double *p) {
        const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double2 t = __ldg(q + i);
            v[2 * i] = t.x; v[2 * i + 1] = t.y;
        }
    }
};

// explicitly rounded, so that every mode evaluates it identically
template <typename T>
__device__ __forceinline__ T zone_phi(const T *__restrict__ ax, const T (&s)[6]) {
    AxisRow<T> a;
    a.load(ax);
    const T s3 = s[3] + s[3], s4 = s[4] + s[4], s5 = s[5] + s[5];
    T p[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const T x = a.v[3 * m], y = a.v[3 * m + 1], z = a.v[3 * m + 2];
        const T t1 = rfma(z, s4, rfma(y, s5, rmul(x, s[0])));   // x s11 + 2 y s12 + 2 z s13
        const T t2 = rfma(z, s3, rmul(y, s[1]));               // y s22 + 2 z s23
        p[m] = rfma(rmul(z, s[2]), z, rfma(y, t2, rmul(x, t1)));
    }
    const T p2 = ((s[0] + s[1]) + s[2]) - p[0] - p[1];
    return rfma(p[0], p[0], rfma(p[1], p[1], rmul(p2, p2)));
}

// FP32: the hardware logarithm (relative error ~1e-7, inside the decision margin the parity
// tests allow); FP64: the correctly rounded library logarithm, as the oracle
__device__ __forceinline__ float log_t(float x) { return __logf(x); }
__device__ __forceinline__ double log_t(double x) { return log(x); }

// Shared-memory list of a CTA's trials that change the orientation (elastic modes):
// the old and new orientation, the acceptance draw, the owning thread and slot with
// the bond-count change, and (flat kernel) the site's stress or strain.
template <typename T, bool SIG, int CTA>
struct SweepList {
    T sig[SIG ? 6 : 1][SIG ? 4 * CTA : 1];
    uint32_t qq[4 * CTA];    // q | q_new << 16
    uint32_t r1[4 * CTA];
    uint16_t own[4 * CTA];   // lane << 2 | slot, bond change + 8 in bits 8..11
    uint8_t acc[4 * CTA];    // decision by (thread, slot)
    unsigned nacc, done;           // acceptances of the CTA; warps finished
};

// warp-aggregated reservation of n entries: returns this lane's first index
__device__ __forceinline__ unsigned warp_reserve(unsigned *counter, int n, int lane) {
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    unsigned base = 0;
    if (lane == 31 && total) base = atomicAdd(counter, (unsigned)total);
    return __shfl_sync(FULL, base, 31) + (unsigned)(incl - n);
}

// The draws of the colour's four sites of block (bx, by, bz), rnd[i] = (trial word,
// acceptance word) of slot i (slots in increasing local corner index).  One
// Philox4x32-10 block per block and colour: counter (index of the block's origin
// site, Monte Carlo step, replica, 2 + colour), key (seed lo, seed hi); word i
// belongs to slot i.  Neighbour trials take the acceptance word from the same
// word w, as the low half of 6 w (the high half picks the neighbour); trials over
// all orientations take it from a second block, counter word 3 = 4 + colour.
// One-replica sweeps (ONE) take the round keys from the kernel argument (rk).
template <int COL, bool ONE>
__device__ __forceinline__ void block_draws(const Replica &R, const uint32_t (&rk)[20], int trial, int bx, int by,
                                            int bz, uint32_t mcs, uint2 (&rnd)[4]) {
    const uint32_t s0 = 2u * ((uint32_t)bx + (uint32_t)R.nx * ((uint32_t)by + (uint32_t)R.ny * (uint32_t)bz));
    const uint4 w = ONE ? philox4_rk(s0, mcs, R.replica, 2u + COL, rk) : philox4(s0, mcs, R.replica, 2u + COL, R.key0, R.key1);
    if (trial == 0) {
        rnd[0] = make_uint2(w.x, 6u * w.x);
        rnd[1] = make_uint2(w.y, 6u * w.y);
        rnd[2] = make_uint2(w.z, 6u * w.z);
        rnd[3] = make_uint2(w.w, 6u * w.w);
    } else {
        const uint4 v = ONE ? philox4_rk(s0, mcs, R.replica, 4u + COL, rk) : philox4(s0, mcs, R.replica, 4u + COL, R.key0, R.key1);
        rnd[0] = make_uint2(w.x, v.x);
        rnd[1] = make_uint2(w.y, v.y);
        rnd[2] = make_uint2(w.z, v.z);
        rnd[3] = make_uint2(w.w, v.w);
    }
}

// The colour's four trials of a block: current and proposed orientation and the
// bond-count change dE = (like bonds lost) - (like bonds gained), zero when the
// proposal keeps the orientation.  O is the block's own quad of the other colour,
// N its -x, +x, -y, +y, -z, +z neighbours' quads of the other colour.
// halves ia of a and ib of b (16-bit orientations of uint2 quads) as one 32-bit pair
__device__ __forceinline__ uint32_t quad_pair(const uint2 &a, int ia, const uint2 &b, int ib) {
    const uint32_t wa = ia < 2 ? a.x : a.y, wb = ib < 2 ? b.x : b.y;
    const uint32_t sel = ((ia & 1) ? 0x32u : 0x10u) | ((ib & 1) ? 0x7600u : 0x5400u);
    return __byte_perm(wa, wb, sel);
}

// number of halves of x that are not zero, per half (0 or 1 each)
__device__ __forceinline__ uint32_t nonzero2(uint32_t x) { return __vminu2(x, 0x00010001u); }

template <int COL>
__device__ __forceinline__ void block_trials(int trial, int nq, const uint2 &mine, const uint2 &O,
                                             const uint2 (&N)[6], const uint2 (&rnd)[4], uint16_t (&q)[4],
                                             uint16_t (&qn)[4], int (&dE)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int L = slot_local(4 * COL + i);
        const int lx = L & 1, ly = (L >> 1) & 1, lz = L >> 2;
        // the six neighbours -x, +x, -y, +y, -z, +z as three pairs of 16-bit halves
        const uint32_t P0 = quad_pair(lx ? O : N[0], i, lx ? N[1] : O, i);
        const uint32_t P1 = quad_pair(ly ? O : N[2], i ^ 1, ly ? N[3] : O, i ^ 1);
        const uint32_t P2 = quad_pair(lz ? O : N[4], i ^ 2, lz ? N[5] : O, i ^ 2);
        const uint32_t qo = quad_get(mine, i);
        uint32_t qnew;
        if (trial == 0) {
            const uint32_t k = __umulhi(rnd[i].x, 6u);   // neighbour k: pair k / 2, half k % 2
            const uint32_t w = k < 2 ? P0 : k < 4 ? P1 : P2;
            qnew = (k & 1) ? w >> 16 : w & 0xffffu;
        } else {
            qnew = __umulhi(rnd[i].x, (uint32_t)nq);
        }
        // dE = (neighbours equal to q) - (neighbours equal to q_new) = (halves differing from
        // q_new) - (halves differing from q), counted per half (at most 3 each) and then summed
        const uint32_t Qo = qo * 0x00010001u, Qn = qnew * 0x00010001u;
        const uint32_t So = nonzero2(P0 ^ Qo) + nonzero2(P1 ^ Qo) + nonzero2(P2 ^ Qo);
        const uint32_t Sn = nonzero2(P0 ^ Qn) + nonzero2(P1 ^ Qn) + nonzero2(P2 ^ Qn);
        const uint32_t U = Sn + 0x00030003u - So;   // per half in 0..6: no borrow between halves
        q[i] = (uint16_t)qo;
        qn[i] = (uint16_t)qnew;
        dE[i] = (int)((U * 0x00010001u) >> 16) - 6;
    }
}

// a replica's scale in the kernel's precision (FP32 kernels read the FP32 copy)
template <typename T>
__device__ __forceinline__ T rep_scale(double d, float f);
template <>
__device__ __forceinline__ float rep_scale<float>(double, float f) { return f; }
template <>
__device__ __forceinline__ double rep_scale<double>(double d, float) { return d; }

// Elastic energy change of a listed trial from the site's stress s (stored forms)
// or, for the recomputing point form, from its strain (then s is overwritten with
// the stress the stress pass would form).
template <typename T, int MODE, bool RECOMP>
__device__ __forceinline__ T trial_dhe(const SweepArgs<T> &a, const Replica &R, uint32_t q, uint32_t qn, T (&s)[6]) {
    if (MODE == SWEEP_POINT) {
        if (RECOMP) {
            T e6[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) e6[k] = s[k];
            Row24<T> rw;
            rw.load(a.ctab + 24ll * q);
            hooke21<T>(rw.v, e6, s);
        }
        return rep_scale<T>(R.lam_sd_half, R.lam_sd_half_f) * (zone_phi<T>(a.atab + 8ll * q, s) - zone_phi<T>(a.atab + 8ll * qn, s));
    }
    // constant strain: e (stored forms: S'(q) s) held fixed, 1/2 (e.C'(q_new)e - e.C'(q)e)
    T e6[6], sn[6], so[6];
    if (RECOMP) {
#pragma unroll
        for (int k = 0; k < 6; ++k) e6[k] = s[k];
    } else {
        Row24<T> rw;
        rw.load(a.stab + 24ll * q);
        hooke21<T>(rw.v, s, e6);
    }
    {
        Row24<T> rw;
        rw.load(a.ctab + 24ll * qn);
        hooke21<T>(rw.v, e6, sn);
    }
    {
        Row24<T> rw;
        rw.load(a.ctab + 24ll * q);
        hooke21<T>(rw.v, e6, so);
    }
    T d = T(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) d = rfma(e6[k], sn[k] - so[k], d);
    return T(0.5) * rep_scale<T>(R.lam, R.lam_f) * d;
}

// Metropolis decision (Eq. 5): the integer threshold table when the elastic term
// vanishes, otherwise H <= -kT ln u with u = (r1 + 1/2) 2^-32.
template <typename T>
__device__ __forceinline__ bool metropolis(const SweepArgs<T> &a, int dE, T dHe, uint32_t r1) {
    if (dHe == T(0)) return dE <= 0 || (unsigned long long)r1 < __ldg(a.thr + dE);
    const T H = rfma(a.J, (T)dE, dHe);
    const T u01 = ((T)r1 + T(0.5)) * T(2.3283064365386963e-10);
    const T t = a.kT > T(0) ? -a.kT * log_t(u01) : T(0);
    return H <= t;
}

// ---------------------------------------------------------------------------
// mbarrier and asynchronous-copy primitives (inline PTX)
// ---------------------------------------------------------------------------
constexpr long long WAIT_NS = 1000000000ll;      // a wait not over after 1 s is a failure
constexpr int WAIT_POLLS = 1 << 24;              // backstop on the number of polls
constexpr int DRAIN_WAITS = 20;                  // further limits a timed-out CTA waits for its copy

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long *b, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}
// wait for the phase of the given parity to complete; false after the time limit
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity) {
    if (mbar_test(b, parity)) return true;
    const long long t0 = global_ns();
    for (int i = 0; i < WAIT_POLLS; ++i) {
        if (mbar_test(b, parity)) return true;
        if (global_ns() - t0 > WAIT_NS) break;
    }
    return false;
}
// The stress is read once per half sweep: its lines are marked evict-first in L2, so that
// the 201 MB stream does not push the spin field (33.5 MB, read by every half sweep) out.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, unsigned long long *b) {
    asm volatile(
        "{\n\t.reg .b64 pol;\n\t"
        "createpolicy.fractional.L2::evict_first.b64 pol, 1.0;\n\t"
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], pol;\n\t}" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(b))
        : "memory");
}
// ---------------------------------------------------------------------------
// Flat kernel: one CTA per tile.  With the stored stress, thread 0 starts a bulk
// copy of the tile's stress of the colour into shared memory as the CTA begins;
// only the listed trials read it, after the threads' own loads and arithmetic.
// ---------------------------------------------------------------------------
template <typename T, bool STORED, int CTA>
struct FlatSmem;
template <typename T, int CTA>
struct FlatSmem<T, false, CTA> {
    SweepList<T, true, CTA> list;
};
template <typename T, int CTA>
struct FlatSmem<T, true, CTA> {
    T sig[6][4 * CTA];
    SweepList<T, false, CTA> list;
    unsigned long long bar;
};

// resident CTAs per SM the kernels are compiled for (measured on the 256^3 workload: six FP32
// one-point-zone CTAs fit registers and shared memory but sweep slower than five)
template <typename T, int MODE, bool RECOMP, int CTA>
__host__ __device__ constexpr int flat_min_ctas() {
    return split_of<CTA>() * (sizeof(T) == 8 ? 2
                    : RECOMP ? 3
                    : MODE == SWEEP_ZONE_LIST ? 4
                    : 5);
}

// ONE: a single replica, whose descriptor is read from the kernel argument (no dependent
// loads before the tile's copy and spin loads can start).  MARGIN: also write each elastic
// trial's (H - t) / max(1, |t|) to a.margin (a diagnostic form; the decisions are the same).
template <typename T, int MODE, bool RECOMP, int COL, bool ONE, bool MARGIN = false, int CTA = SWEEP_CTA>
__global__ void __launch_bounds__(CTA, flat_min_ctas<T, MODE, RECOMP, CTA>())
    k_sweep(const __grid_constant__ SweepArgs<T> a) {
    constexpr int SPLIT = split_of<CTA>();
    constexpr bool ELASTIC = MODE == SWEEP_POINT || MODE == SWEEP_STRAIN;   // a point-zone elastic term
    constexpr bool STORED = ELASTIC && !RECOMP;                               // ... from the stored stress
    constexpr bool LIST = MODE == SWEEP_ZONE_LIST;
    extern __shared__ __align__(128) unsigned char sweep_smem[];
    FlatSmem<T, STORED, CTA> &fs = *reinterpret_cast<FlatSmem<T, STORED, CTA> *>(sweep_smem);
    auto &sl = fs.list;
    // the red half sweep follows the stress pass: its CTAs take the tiles in reverse order, so
    // that the first to run read the stress the pass wrote last, still in L2
    const int bid = COL == 0 ? (int)gridDim.x - 1 - (int)blockIdx.x : (int)blockIdx.x;
    const int tile = bid / SPLIT;
    const int r = ONE ? 0 : __ldg(a.cta_rep + tile);
    const Replica &R = ONE ? a.rep0 : a.reps[r];
    const int tid = threadIdx.x, lane = tid & 31;
    const int t0 = (tile - R.cta_off) * BLOCK_THREADS + (bid % SPLIT) * CTA;
    if (t0 >= R.nblk) return;  // the empty part of a replica's last tile
    const int blk = t0 + tid;  // block within the replica
    if (ELASTIC) {
        if (tid == 0) {
            sl.nacc = 0;
            sl.done = 0;
            if constexpr (STORED) {
                // the colour's stress of the tile: six components, four values per block, each
                // source a multiple of 16 B in address and size
                const unsigned nb = (unsigned)min(CTA, R.nblk - t0);
                mbar_init(&fs.bar, 1);
                mbar_init_fence();
                if (!a.skip_copy) {
                    mbar_expect_tx(&fs.bar, nb * 24u * (unsigned)sizeof(T));
                    const T *sig = a.sig + 48ll * R.blk_off + 4ll * ((long long)(COL * 6) * R.nblk + t0);
#pragma unroll
                    for (int k = 0; k < 6; ++k)
                        bulk_load(&fs.sig[k][0], sig + 4ll * k * R.nblk, nb * 4u * (unsigned)sizeof(T), &fs.bar);
                }
            }
        }
    }
    int nacc = 0;
    uint4 ent[4];   // zone mode: this thread's trials for the list
    int nent = 0;
    uint16_t out[4] = {0, 0, 0, 0}, qn[4] = {0, 0, 0, 0};
    uint32_t pend = 0;   // elastic modes: slots with a listed trial
    T sg[6][4];          // recompute mode: strain of the colour's four sites
    uint2 rnd[4];
    int dE[4] = {0, 0, 0, 0};
    const bool live = blk < R.nblk;
    if (live) {
        const int nbx = R.nbx, nby = R.nby, nbz = R.nbz;
        int bx, by, bz;
        block_xyz(R, blk, bx, by, bz);
        const int sxy = nbx, sxz = nbx * nby;
        const uint4 *spins = a.spins + R.blk_off;
        const uint2 *q2 = reinterpret_cast<const uint2 *>(spins);
        constexpr int oc = COL ^ 1;
        const uint4 own4 = spins[blk];
        const uint2 mine = COL ? make_uint2(own4.z, own4.w) : make_uint2(own4.x, own4.y);
        const uint2 O = oc ? make_uint2(own4.z, own4.w) : make_uint2(own4.x, own4.y);
        uint2 N[6];
        N[0] = __ldg(q2 + 2 * (blk + (bx == 0 ? nbx - 1 : -1)) + oc);
        N[1] = __ldg(q2 + 2 * (blk + (bx == nbx - 1 ? 1 - nbx : 1)) + oc);
        N[2] = __ldg(q2 + 2 * (blk + (by == 0 ? (nby - 1) * sxy : -sxy)) + oc);
        N[3] = __ldg(q2 + 2 * (blk + (by == nby - 1 ? -(nby - 1) * sxy : sxy)) + oc);
        N[4] = __ldg(q2 + 2 * (blk + (bz == 0 ? (nbz - 1) * sxz : -sxz)) + oc);
        N[5] = __ldg(q2 + 2 * (blk + (bz == nbz - 1 ? -(nbz - 1) * sxz : sxz)) + oc);
        block_draws<COL, ONE>(R, a.rkey, a.trial, bx, by, bz, R.st->mcs, rnd);
        uint16_t q[4];
        block_trials<COL>(a.trial, a.nq, mine, O, N, rnd, q, qn, dE);
        // recompute mode: the cell's displacement gradients, formed at the first listed trial
        CellGrad<T> g;
        T ebv[6];
        bool have_g = false;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            out[i] = q[i];
            if (qn[i] == q[i]) continue;
            const int L = slot_local(4 * COL + i);
            const int lx = L & 1, ly = (L >> 1) & 1, lz = L >> 2;
            if (LIST) {
                const uint32_t x = 2u * bx + lx, y = 2u * by + ly, z = 2u * bz + lz;
                const uint4 en = make_uint4(x + (uint32_t)R.nx * (y + (uint32_t)R.ny * z), (uint32_t)r,
                                            (uint32_t)qn[i] | ((uint32_t)q[i] << 16), rnd[i].y);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (j == nent) ent[j] = en;
                ++nent;
                continue;
            }
            if (!ELASTIC) {
                if (dE[i] <= 0 || (unsigned long long)rnd[i].y < __ldg(a.thr + dE[i])) {
                    out[i] = qn[i];
                    ++nacc;
                }
                continue;
            }
            pend |= 1u << i;
            if (RECOMP) {
                if (!have_g) {
                    // the cell's eight corner displacements, as the stress pass reads them
                    const T *u = a.u + 3 * R.blk_off;
                    T uc[8][3];
#pragma unroll
                    for (int K = 0; K < 2; ++K)
#pragma unroll
                        for (int J = 0; J < 2; ++J)
#pragma unroll
                            for (int I = 0; I < 2; ++I) {
                                const int gi = bx + I == nbx ? 0 : bx + I;
                                const int gj = by + J == nby ? 0 : by + J;
                                const int gk = bz + K == nbz ? 0 : bz + K;
                                const int n = 3 * (gi + nbx * (gj + nby * gk));
#pragma unroll
                                for (int d = 0; d < 3; ++d) uc[corner(I, J, K)][d] = __ldg(u + n + d);
                            }
                    cell_gradients<T>(uc, g);
                    load_ebar<T>(R.st, ebv);
                    have_g = true;
                }
                T er[6];
                point_strain<T>(g, ebv, lx, ly, lz, er);
#pragma unroll
                for (int k = 0; k < 6; ++k) sg[k][i] = er[k];
            }
        }
    }

    unsigned dacc = 0;   // elastic forms: acceptances decided by this thread
    if (ELASTIC) {
        // each warp lists its pending trials in its own region of the list: slot 0 trials of
        // lanes 0..31, then slot 1, ...
        const unsigned below = (1u << lane) - 1u;
        const int wb = (tid >> 5) * 128;
        unsigned n = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool pi = (pend >> i) & 1u;
            const unsigned m = __ballot_sync(FULL, pi);
            if (pi) {
                const unsigned idx = wb + n + __popc(m & below);
                if constexpr (!STORED) {
#pragma unroll
                    for (int k = 0; k < 6; ++k) sl.sig[k][idx] = sg[k][i];
                }
                sl.qq[idx] = (uint32_t)out[i] | ((uint32_t)qn[i] << 16);
                sl.r1[idx] = rnd[i].y;
                sl.own[idx] = (uint16_t)((lane << 2 | i) | ((dE[i] + 8) << 8));
            }
            n += __popc(m);
        }
        bool ok = true;
        if constexpr (STORED)
            if (tid == 0) ok = mbar_wait(&fs.bar, 0u);   // the tile's stress has landed
        if (__syncthreads_or(!ok)) {
            // The copy did not complete within the limit: report it and decide nothing.  No bulk
            // copy may still be writing this CTA's shared memory when the CTA returns, or it
            // would land in the shared memory of whichever CTA the SM runs next.  Either no copy
            // was started (the injected fault, skip_copy), or thread 0 keeps waiting until the
            // copy's mbarrier phase completes, which happens exactly when all its bytes have
            // landed.  A copy of valid device memory always completes; only if it has not after
            // DRAIN_WAITS further limits does the CTA return with it outstanding, and then it
            // records wait_timeout = 2, which the host reports as a lost context (the handle
            // refuses every later call).
            if (tid == 0) {
                atomicExch(&R.st->wait_timeout, 1);
                if constexpr (STORED) {
                    if (!a.skip_copy) {
                        bool landed = false;
                        for (int k = 0; k < DRAIN_WAITS && !landed; ++k) landed = mbar_wait(&fs.bar, 0u);
                        if (!landed) atomicExch(&R.st->wait_timeout, 2);
                    }
                }
            }
            return;
        }
        // the warp's listed trials, evaluated densely by its lanes
        for (unsigned e = lane; e < n; e += 32) {
            const uint32_t qq = sl.qq[wb + e], ow = sl.own[wb + e];
            const int site = wb + (int)(ow & 0x7fu);   // thread << 2 | slot
            T s[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                if constexpr (STORED)
                    s[k] = fs.sig[k][site];
                else
                    s[k] = sl.sig[k][wb + e];
            }
            const T dHe = trial_dhe<T, MODE, RECOMP>(a, R, qq & 0xffffu, qq >> 16, s);
            const bool acc = metropolis<T>(a, (int)(ow >> 8) - 8, dHe, sl.r1[wb + e]);
            if constexpr (MARGIN) {
                // the trial's site: block t0 + (owning thread), slot ow & 3 of the colour
                int bx, by, bz;
                block_xyz(R, t0 + (site >> 2), bx, by, bz);
                const int L = slot_local(4 * COL + (int)(ow & 3u));
                const long long x = 2 * bx + (L & 1), y = 2 * by + ((L >> 1) & 1), z = 2 * bz + (L >> 2);
                const T H = rfma(a.J, (T)((int)(ow >> 8) - 8), dHe);
                const T u01 = ((T)sl.r1[wb + e] + T(0.5)) * T(2.3283064365386963e-10);
                const T t = a.kT > T(0) ? -a.kT * log_t(u01) : T(0);
                const T den = fabs(t) > T(1) ? fabs(t) : T(1);
                a.margin[x + (long long)R.nx * (y + (long long)R.ny * z)] = (double)((H - t) / den);
            }
            sl.acc[site] = acc ? 1 : 0;
            dacc += acc ? 1u : 0u;
        }
        __syncwarp();
        if (pend) {
            const uint32_t acc4 = *reinterpret_cast<const uint32_t *>(&sl.acc[tid << 2]);   // slots 0..3
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if ((pend & (1u << i)) && ((acc4 >> (8 * i)) & 0xffu)) {
                    out[i] = qn[i];
                    ++nacc;
                }
        }
    }
    if (live && nacc) {
        uint2 w;
        w.x = (uint32_t)out[0] | ((uint32_t)out[1] << 16);
        w.y = (uint32_t)out[2] | ((uint32_t)out[3] << 16);
        reinterpret_cast<uint2 *>(a.spins + R.blk_off)[2 * blk + COL] = w;
    }
    if (LIST) {
        const unsigned first = warp_reserve(a.count, nent, lane);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < nent) a.work[first + j] = ent[j];
        return;
    }
    // a CTA belongs to one replica: one atomic per CTA on that replica's counter (warps of every
    // CTA adding to one address directly would serialise at its L2 slice)
    if constexpr (ELASTIC) {
        // the last warp to finish adds the CTA's acceptances
        const unsigned wt = __reduce_add_sync(FULL, dacc);
        if (lane == 0) {
            if (wt) atomicAdd(&sl.nacc, wt);
            __threadfence_block();
            if (atomicAdd(&sl.done, 1u) == CTA / 32 - 1) {
                __threadfence_block();
                const unsigned c = atomicAdd(&sl.nacc, 0u);
                if (c) atomicAdd(&R.st->accepted, (unsigned long long)c);
            }
        }
        return;
    }
    __shared__ unsigned warp_tot[CTA / 32];
    const unsigned tot = __reduce_add_sync(FULL, (unsigned)nacc);
    if (lane == 0) warp_tot[tid >> 5] = tot;
    __syncthreads();
    if (tid == 0) {
        unsigned c = 0;
#pragma unroll
        for (int w = 0; w < CTA / 32; ++w) c += warp_tot[w];
        if (c) atomicAdd(&R.st->accepted, (unsigned long long)c);
    }
}

template <typename T, int MODE, bool RECOMP, int CTA = SWEEP_CTA>
constexpr size_t flat_smem_bytes() {
    constexpr bool ELASTIC = MODE == SWEEP_POINT || MODE == SWEEP_STRAIN;
    return ELASTIC ? sizeof(FlatSmem<T, !RECOMP, CTA>) : 0;
}

// forms with the 128-thread CTA (a tile split over two CTAs) as a tuning choice
template <int MODE, bool RECOMP>
constexpr bool has_half_cta() {
    return (MODE == SWEEP_POINT && !RECOMP) || MODE == SWEEP_POTTS;
}

template <typename T, int MODE, bool RECOMP, int COL, int CTA>
void launch_flat_cta(const SweepArgs<T> &a, cudaStream_t s) {
    constexpr int SPLIT = split_of<CTA>();
    constexpr size_t smem = flat_smem_bytes<T, MODE, RECOMP, CTA>();
    if (a.nrep == 1)
        k_sweep<T, MODE, RECOMP, COL, true, false, CTA><<<a.nctas * SPLIT, CTA, smem, s>>>(a);
    else
        k_sweep<T, MODE, RECOMP, COL, false, false, CTA><<<a.nctas * SPLIT, CTA, smem, s>>>(a);
}

template <typename T, int MODE, bool RECOMP, int COL>
void launch_flat(const SweepArgs<T> &a, cudaStream_t s) {
    if constexpr (has_half_cta<MODE, RECOMP>()) {
        if (a.cta == 128) {
            launch_flat_cta<T, MODE, RECOMP, COL, 128>(a, s);
            return;
        }
    }
    launch_flat_cta<T, MODE, RECOMP, COL, SWEEP_CTA>(a, s);
}

template <typename T, int MODE, bool RECOMP>
void launch_form(const SweepArgs<T> &a, int colour, cudaStream_t s) {
    if (colour)
        launch_flat<T, MODE, RECOMP, 1>(a, s);
    else
        launch_flat<T, MODE, RECOMP, 0>(a, s);
}

template <typename T, int MODE, bool RECOMP, int CTA>
cudaError_t set_flat_smem_cta() {
    const int bytes = (int)flat_smem_bytes<T, MODE, RECOMP, CTA>();
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_sweep<T, MODE, RECOMP, 0, false, false, CTA>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_sweep<T, MODE, RECOMP, 1, false, false, CTA>, at, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_sweep<T, MODE, RECOMP, 0, true, false, CTA>, at, bytes)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_sweep<T, MODE, RECOMP, 1, true, false, CTA>, at, bytes);
}

template <typename T, int MODE, bool RECOMP>
cudaError_t set_flat_smem() {
    cudaError_t e = set_flat_smem_cta<T, MODE, RECOMP, SWEEP_CTA>();
    if constexpr (has_half_cta<MODE, RECOMP>())
        if (e == cudaSuccess) e = set_flat_smem_cta<T, MODE, RECOMP, 128>();
    return e;
}

}  // namespace

cudaError_t sweep_prepare() {
    cudaError_t e;
    if ((e = set_flat_smem<float, SWEEP_POINT, false>()) != cudaSuccess) return e;
    if ((e = set_flat_smem<float, SWEEP_POINT, true>()) != cudaSuccess) return e;
    if ((e = set_flat_smem<float, SWEEP_STRAIN, false>()) != cudaSuccess) return e;
    if ((e = set_flat_smem<float, SWEEP_STRAIN, true>()) != cudaSuccess) return e;
    if ((e = set_flat_smem<double, SWEEP_POINT, false>()) != cudaSuccess) return e;
    if ((e = set_flat_smem<double, SWEEP_POINT, true>()) != cudaSuccess) return e;
    if ((e = set_flat_smem<double, SWEEP_STRAIN, false>()) != cudaSuccess) return e;
    if ((e = set_flat_smem<double, SWEEP_STRAIN, true>()) != cudaSuccess) return e;
    return cudaSuccess;
}

template <typename T, int MODE, int COL>
void launch_margin_form(const SweepArgs<T> &a, cudaStream_t s) {
    k_sweep<T, MODE, false, COL, true, true><<<a.nctas * split_of<SWEEP_CTA>(), SWEEP_CTA,
                                               flat_smem_bytes<T, MODE, false>(), s>>>(a);
}

template <typename T, int MODE>
cudaError_t set_margin_smem() {
    const int bytes = (int)flat_smem_bytes<T, MODE, false>();
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_sweep<T, MODE, false, 0, true, true>, at, bytes)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_sweep<T, MODE, false, 1, true, true>, at, bytes);
}

template <typename T>
cudaError_t launch_sweep_margin(const SweepArgs<T> &a, int colour, int mode, cudaStream_t s) {
    cudaError_t e;
    if (mode == SWEEP_STRAIN) {
        if ((e = set_margin_smem<T, SWEEP_STRAIN>()) != cudaSuccess) return e;
        if (colour) launch_margin_form<T, SWEEP_STRAIN, 1>(a, s);
        else launch_margin_form<T, SWEEP_STRAIN, 0>(a, s);
    } else {
        if ((e = set_margin_smem<T, SWEEP_POINT>()) != cudaSuccess) return e;
        if (colour) launch_margin_form<T, SWEEP_POINT, 1>(a, s);
        else launch_margin_form<T, SWEEP_POINT, 0>(a, s);
    }
    return cudaGetLastError();
}

template cudaError_t launch_sweep_margin<float>(const SweepArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_sweep_margin<double>(const SweepArgs<double> &, int, int, cudaStream_t);

template <typename T>
cudaError_t launch_sweep(const SweepArgs<T> &a, int colour, int mode, bool recompute, cudaStream_t s) {
    if (mode == SWEEP_POINT && recompute)
        launch_form<T, SWEEP_POINT, true>(a, colour, s);
    else if (mode == SWEEP_POINT)
        launch_form<T, SWEEP_POINT, false>(a, colour, s);
    else if (mode == SWEEP_STRAIN && recompute)
        launch_form<T, SWEEP_STRAIN, true>(a, colour, s);
    else if (mode == SWEEP_STRAIN)
        launch_form<T, SWEEP_STRAIN, false>(a, colour, s);
    else if (mode == SWEEP_ZONE_LIST)
        launch_form<T, SWEEP_ZONE_LIST, false>(a, colour, s);
    else
        launch_form<T, SWEEP_POTTS, false>(a, colour, s);
    return cudaGetLastError();
}

template cudaError_t launch_sweep<float>(const SweepArgs<float> &, int, int, bool, cudaStream_t);
template cudaError_t launch_sweep<double>(const SweepArgs<double> &, int, int, bool, cudaStream_t);

}  // namespace hmc
