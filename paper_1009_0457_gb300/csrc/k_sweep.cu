// Red/black checkerboard half sweep (Sec. "Microstructural Evolution") with the
// Metropolis rule (Eq. 5) on the bond-energy change of the Potts Hamiltonian
// (Eq. 4, bonds counted once, 6 neighbours, periodic) plus the one-point
// constant-traction zone shift (Eqs. 6-8 and 13) from the stored stress, or its
// constant-strain reading.
//
// One thread per 2x2x2 block: it draws the trials of the block's four sites of
// the sweep's colour.  A CTA covers 256 blocks of one replica of the batch.
// Loads per block: the block's 16 B of spins, the other colour's 8 B quad of
// the six face neighbours (cache hits: every quad is some other thread's own),
// and six 16 B stress vectors (FP32).  Writes: the colour's 8 B quad when a site
// changed.  Same-colour sites share no neighbour, so the in-place update is race
// free.  Two sites of a colour share one Philox4x32-10 block (four words, two
// per site).
//
// With an elastic term, the trials that change the orientation (a minority:
// interior sites copy their own orientation) are listed in shared memory with
// their stress, and the CTA's threads then evaluate the listed trials densely,
// so that the zone energies and the logarithm of the Metropolis threshold run
// with full warps rather than on the few lanes whose site needs them.
//
// With the 27-point zone the sweep only lists its non-trivial trials (site,
// replica, old and new orientation, the acceptance draw) in global memory with
// one atomic per warp; the zone kernel decides them.
#include "hmc_device.cuh"

namespace hmc {

namespace {

constexpr unsigned FULL = 0xffffffffu;

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    float v[4];
    __device__ __forceinline__ void load(const float *p) {
        const float4 t = __ldcs(reinterpret_cast<const float4 *>(p));  // streamed once per sweep
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
};
template <>
struct Vec4<double> {
    double v[4];
    __device__ __forceinline__ void load(const double *p) {
        const double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
        const double2 b = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};

// Phi(q; sigma) = sum over the three crystal axes of (a_m . sigma . a_m)^2, from
// the Voigt weight vectors of the axes.  For one cubic material the zone energy
// w(q) = 1/2 sigma.S'(q).sigma = 1/2 [S12 tr^2 + S44/2 |sigma|^2 + s_d Phi(q)], so
// w(q_old) - w(q_new) = s_d / 2 (Phi(q_old) - Phi(q_new)).
template <typename T>
struct Row20;
template <>
struct Row20<float> {
    float v[20];
    __device__ __forceinline__ void load(const float *p) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float4 t = __ldg(q + i);
            v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
        }
    }
};
template <>
struct Row20<double> {
    double v[20];
    __device__ __forceinline__ void load(const double *p) {
        const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double2 t = __ldg(q + i);
            v[2 * i] = t.x; v[2 * i + 1] = t.y;
        }
    }
};

// explicitly rounded, so that every mode evaluates it identically
template <typename T>
__device__ __forceinline__ T zone_phi(const T *__restrict__ w, const T (&s)[6]) {
    Row20<T> r;
    r.load(w);
    T acc = T(0);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        T p = rmul(r.v[6 * m], s[0]);
#pragma unroll
        for (int k = 1; k < 6; ++k) p = rfma(r.v[6 * m + k], s[k], p);
        acc = rfma(p, p, acc);
    }
    return acc;
}

// FP32: the hardware logarithm (relative error ~1e-7, inside the decision margin the parity
// tests allow); FP64: the correctly rounded library logarithm, as the oracle
__device__ __forceinline__ float log_t(float x) { return __logf(x); }
__device__ __forceinline__ double log_t(double x) { return log(x); }

// Shared-memory list of a CTA's trials that change the orientation (elastic modes):
// the site's stress (stored mode) or strain (recompute mode), the old and new
// orientation, the bond-count change, the acceptance draw and the owning thread and slot.
template <typename T>
struct SweepList {
    T sig[6][4 * BLOCK_THREADS];
    uint32_t qq[4 * BLOCK_THREADS];    // q | q_new << 16
    uint32_t r1[4 * BLOCK_THREADS];
    uint32_t own[4 * BLOCK_THREADS];   // thread << 2 | slot, bond change + 8 in bits 16..23
    uint8_t acc[4 * BLOCK_THREADS];    // decision by (thread, slot)
    unsigned count;
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

template <typename T, int MODE, bool RECOMP>
__global__ void __launch_bounds__(BLOCK_THREADS, (sizeof(T) == 4 ? 4 : 2)) k_sweep(SweepArgs<T> a, int colour) {
    constexpr bool ELASTIC = MODE == SWEEP_POINT || MODE == SWEEP_STRAIN;   // a point-zone elastic term
    constexpr bool STORED = ELASTIC && !RECOMP;                               // ... from the stored stress
    constexpr bool LIST = MODE == SWEEP_ZONE_LIST;
    extern __shared__ __align__(16) unsigned char sweep_smem[];
    SweepList<T> &sl = *reinterpret_cast<SweepList<T> *>(sweep_smem);
    const int r = __ldg(a.cta_rep + blockIdx.x);
    const Replica &R = a.reps[r];
    const int tid = threadIdx.x, lane = tid & 31;
    const int blk = (blockIdx.x - R.cta_off) * BLOCK_THREADS + tid;  // block within the replica
    if (ELASTIC) {
        if (tid == 0) sl.count = 0;
        __syncthreads();
    }
    int nacc = 0;
    uint4 ent[4];   // zone mode: this thread's trials for the list
    int nent = 0;
    uint16_t out[4] = {0, 0, 0, 0}, qnew[4] = {0, 0, 0, 0};
    uint32_t pend = 0;   // elastic modes: slots with a listed trial
    T sg[6][4];          // elastic modes: stress (stored) or strain (recompute) of the colour's four sites
    uint2 rnd[4];
    int dEs[4] = {0, 0, 0, 0};
    const bool live = blk < R.nblk;
    if (live) {
        const int nbx = R.nbx, nby = R.nby, nbz = R.nbz;
        const int bx = blk % nbx, rr = blk / nbx;
        const int by = rr % nby, bz = rr / nby;
        const int sxy = nbx, sxz = nbx * nby;
        const int bxm = blk + (bx == 0 ? nbx - 1 : -1), bxp = blk + (bx == nbx - 1 ? 1 - nbx : 1);
        const int bym = blk + (by == 0 ? (nby - 1) * sxy : -sxy);
        const int byp = blk + (by == nby - 1 ? -(nby - 1) * sxy : sxy);
        const int bzm = blk + (bz == 0 ? (nbz - 1) * sxz : -sxz);
        const int bzp = blk + (bz == nbz - 1 ? -(nbz - 1) * sxz : sxz);
        const uint4 *spins = a.spins + R.blk_off;
        const uint2 *q2 = reinterpret_cast<const uint2 *>(spins);
        const int oc = colour ^ 1;
        const uint4 own4 = spins[blk];
        const uint2 mine = colour ? make_uint2(own4.z, own4.w) : make_uint2(own4.x, own4.y);
        const uint2 O = oc ? make_uint2(own4.z, own4.w) : make_uint2(own4.x, own4.y);
        const uint2 Oxm = __ldg(q2 + 2 * bxm + oc), Oxp = __ldg(q2 + 2 * bxp + oc);
        const uint2 Oym = __ldg(q2 + 2 * bym + oc), Oyp = __ldg(q2 + 2 * byp + oc);
        const uint2 Ozm = __ldg(q2 + 2 * bzm + oc), Ozp = __ldg(q2 + 2 * bzp + oc);
        if (STORED) {
            const T *sig = a.sig + 48ll * R.blk_off;
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                Vec4<T> t;
                t.load(sig + 4ll * ((long long)(colour * 6 + k) * R.nblk + blk));
#pragma unroll
                for (int i = 0; i < 4; ++i) sg[k][i] = t.v[i];
            }
        }
        const uint32_t mcs = R.st->mcs;
        // Two Philox blocks per thread.  The colour's sites pair up as (even-x site, its
        // partner at x+1, y^1): red slots (0, 1) and (3, 2), black (1, 0) and (2, 3),
        // leader first; the leader takes words 0 and 1, the partner words 2 and 3.
        {
            const int la = colour ? 1 : 0, pa = colour ? 0 : 1, lb = colour ? 2 : 3;
            const int LA = slot_local(4 * colour + la), LB = slot_local(4 * colour + lb);
            const uint32_t xa = 2u * bx + (LA & 1), ya = 2u * by + ((LA >> 1) & 1), za = 2u * bz + (LA >> 2);
            const uint32_t xb = 2u * bx + (LB & 1), yb = 2u * by + ((LB >> 1) & 1), zb = 2u * bz + (LB >> 2);
            const uint4 wa = philox4(xa + (uint32_t)R.nx * (ya + (uint32_t)R.ny * za), mcs, R.replica, 0u, R.key0,
                                     R.key1);
            const uint4 wb = philox4(xb + (uint32_t)R.nx * (yb + (uint32_t)R.ny * zb), mcs, R.replica, 0u, R.key0,
                                     R.key1);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                rnd[i] = i == la ? make_uint2(wa.x, wa.y)
                         : i == pa ? make_uint2(wa.z, wa.w)
                         : i == lb ? make_uint2(wb.x, wb.y)
                                   : make_uint2(wb.z, wb.w);
        }
        // recompute mode: the cell's displacement gradients, formed at the first listed trial
        CellGrad<T> g;
        T ebv[6];
        bool have_g = false;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int L = slot_local(4 * colour + i);
            const int lx = L & 1, ly = (L >> 1) & 1, lz = L >> 2;
            const uint16_t q = quad_get(mine, i);
            uint16_t nb[6];
            nb[0] = quad_get(lx ? O : Oxm, i);
            nb[1] = quad_get(lx ? Oxp : O, i);
            nb[2] = quad_get(ly ? O : Oym, i ^ 1);
            nb[3] = quad_get(ly ? Oyp : O, i ^ 1);
            nb[4] = quad_get(lz ? O : Ozm, i ^ 2);
            nb[5] = quad_get(lz ? Ozp : O, i ^ 2);
            const uint2 rn = rnd[i];
            uint16_t qn;
            if (a.trial == 0) {
                const uint32_t k = __umulhi(rn.x, 6u);
                qn = nb[0];
#pragma unroll
                for (int j = 1; j < 6; ++j)
                    if (k == (uint32_t)j) qn = nb[j];
            } else {
                qn = (uint16_t)__umulhi(rn.x, (uint32_t)a.nq);
            }
            out[i] = q;
            qnew[i] = qn;
            if (qn == q) continue;
            if (LIST) {
                const uint32_t x = 2u * bx + lx, y = 2u * by + ly, z = 2u * bz + lz;
                const uint4 en = make_uint4(x + (uint32_t)R.nx * (y + (uint32_t)R.ny * z), (uint32_t)r,
                                            (uint32_t)qn | ((uint32_t)q << 16), rn.y);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (j == nent) ent[j] = en;
                ++nent;
                continue;
            }
            int dE = 0;
#pragma unroll
            for (int j = 0; j < 6; ++j) dE += (nb[j] == q) - (nb[j] == qn);
            if (!ELASTIC) {
                if (dE <= 0 || (unsigned long long)rn.y < __ldg(a.thr + dE)) {
                    out[i] = qn;
                    ++nacc;
                }
                continue;
            }
            dEs[i] = dE;
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

    if (ELASTIC) {
        // list the pending trials (every lane of the warp takes part in the reservation)
        unsigned idx = warp_reserve(&sl.count, __popc(pend), lane);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (pend & (1u << i)) {
#pragma unroll
                for (int k = 0; k < 6; ++k) sl.sig[k][idx] = sg[k][i];
                sl.qq[idx] = (uint32_t)out[i] | ((uint32_t)qnew[i] << 16);
                sl.r1[idx] = rnd[i].y;
                sl.own[idx] = (uint32_t)(tid << 2 | i) | ((uint32_t)(dEs[i] + 8) << 16);
                ++idx;
            }
        __syncthreads();
        // the listed trials, evaluated densely by all threads of the CTA
        const unsigned n = sl.count;
        const T lam_sd_half = (T)R.lam_sd_half;
        for (unsigned e = tid; e < n; e += BLOCK_THREADS) {
            const uint32_t qq = sl.qq[e], ow = sl.own[e];
            const uint32_t q = qq & 0xffffu, qn = qq >> 16, r1 = sl.r1[e];
            const int dE = (int)((ow >> 16) & 0xffu) - 8;
            T s[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) s[k] = sl.sig[k][e];
            T dHe = T(0);
            if (MODE == SWEEP_POINT) {
                if (RECOMP) {
                    // the entry holds the strain: the stress with the site's stiffness, as the stress pass forms it
                    T e6[6];
#pragma unroll
                    for (int k = 0; k < 6; ++k) e6[k] = s[k];
                    Row24<T> rw;
                    rw.load(a.ctab + 24ll * q);
                    hooke21<T>(rw.v, e6, s);
                }
                dHe = lam_sd_half * (zone_phi<T>(a.wtab + 20ll * q, s) - zone_phi<T>(a.wtab + 20ll * qn, s));
            } else {
                // constant strain: e (stored mode: S'(q) s) held fixed, 1/2 (e.C'(q_new)e - e.C'(q)e)
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
                dHe = T(0.5) * (T)R.lam * d;
            }
            bool acc;
            if (dHe == T(0)) {
                acc = dE <= 0 || (unsigned long long)r1 < __ldg(a.thr + dE);
            } else {
                const T H = rfma(a.J, (T)dE, dHe);
                const T u01 = ((T)r1 + T(0.5)) * T(2.3283064365386963e-10);
                const T t = a.kT > T(0) ? -a.kT * log_t(u01) : T(0);
                acc = H <= t;
            }
            sl.acc[ow & 0xffffu] = acc ? 1 : 0;
        }
        __syncthreads();
        if (pend) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if ((pend & (1u << i)) && sl.acc[tid << 2 | i]) {
                    out[i] = qnew[i];
                    ++nacc;
                }
        }
    }
    if (live && nacc) {
        uint2 w;
        w.x = (uint32_t)out[0] | ((uint32_t)out[1] << 16);
        w.y = (uint32_t)out[2] | ((uint32_t)out[3] << 16);
        reinterpret_cast<uint2 *>(a.spins + R.blk_off)[2 * blk + colour] = w;
    }
    if (LIST) {
        const unsigned first = warp_reserve(a.count, nent, lane);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < nent) a.work[first + j] = ent[j];
        return;
    }
    // a CTA belongs to one replica: warp totals go to that replica's counter
    const unsigned tot = __reduce_add_sync(FULL, (unsigned)nacc);
    if (lane == 0 && tot) atomicAdd(&R.st->accepted, (unsigned long long)tot);
}

template <typename T, int MODE, bool RECOMP>
void launch_one(const SweepArgs<T> &a, int colour, cudaStream_t s) {
    constexpr bool ELASTIC = MODE == SWEEP_POINT || MODE == SWEEP_STRAIN;
    k_sweep<T, MODE, RECOMP><<<a.nctas, BLOCK_THREADS, ELASTIC ? sizeof(SweepList<T>) : 0, s>>>(a, colour);
}

template <typename T, int MODE, bool RECOMP>
cudaError_t set_smem() {
    return cudaFuncSetAttribute(k_sweep<T, MODE, RECOMP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(SweepList<T>));
}

}  // namespace

cudaError_t sweep_prepare() {
    cudaError_t e;
    if ((e = set_smem<float, SWEEP_POINT, false>()) != cudaSuccess) return e;
    if ((e = set_smem<float, SWEEP_POINT, true>()) != cudaSuccess) return e;
    if ((e = set_smem<float, SWEEP_STRAIN, false>()) != cudaSuccess) return e;
    if ((e = set_smem<float, SWEEP_STRAIN, true>()) != cudaSuccess) return e;
    if ((e = set_smem<double, SWEEP_POINT, false>()) != cudaSuccess) return e;
    if ((e = set_smem<double, SWEEP_POINT, true>()) != cudaSuccess) return e;
    if ((e = set_smem<double, SWEEP_STRAIN, false>()) != cudaSuccess) return e;
    return set_smem<double, SWEEP_STRAIN, true>();
}

template <typename T>
cudaError_t launch_sweep(const SweepArgs<T> &a, int colour, int mode, bool recompute, cudaStream_t s) {
    if (mode == SWEEP_POINT && recompute)
        launch_one<T, SWEEP_POINT, true>(a, colour, s);
    else if (mode == SWEEP_POINT)
        launch_one<T, SWEEP_POINT, false>(a, colour, s);
    else if (mode == SWEEP_STRAIN && recompute)
        launch_one<T, SWEEP_STRAIN, true>(a, colour, s);
    else if (mode == SWEEP_STRAIN)
        launch_one<T, SWEEP_STRAIN, false>(a, colour, s);
    else if (mode == SWEEP_ZONE_LIST)
        launch_one<T, SWEEP_ZONE_LIST, false>(a, colour, s);
    else
        launch_one<T, SWEEP_POTTS, false>(a, colour, s);
    return cudaGetLastError();
}

template cudaError_t launch_sweep<float>(const SweepArgs<float> &, int, int, bool, cudaStream_t);
template cudaError_t launch_sweep<double>(const SweepArgs<double> &, int, int, bool, cudaStream_t);

}  // namespace hmc
