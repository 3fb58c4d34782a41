// Red/black checkerboard half sweep (Sec. "Microstructural Evolution") with the
// Metropolis rule (Eq. 5) on the bond-energy change of the Potts Hamiltonian
// (Eq. 4, bonds counted once, 6 neighbours, periodic) plus the one-point
// constant-traction zone shift (Eqs. 6-8 and 13) from the stored stress, or its
// constant-strain reading.
//
// One thread per 2x2x2 block: it tries the block's four sites of the sweep's
// colour.  A CTA covers 256 blocks of one replica of the batch.  Loads per
// block: the block's 16 B of spins, the other colour's 8 B quad of the six face
// neighbours (cache hits: every quad is some other thread's own), and six 16 B
// stress vectors (FP32).  Writes: the colour's 8 B quad when a site changed.
// Same-colour sites share no neighbour, so the in-place update is race free.
//
// With the 27-point zone the sweep only lists its non-trivial trials (site,
// replica, old and new orientation, the acceptance draw) with one atomic per
// warp; the zone kernel decides them.
#include "hmc_device.cuh"

namespace hmc {

namespace {

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

template <typename T>
__device__ __forceinline__ T zone_phi(const T *__restrict__ w, const T (&s)[6]) {
    Row20<T> r;
    r.load(w);
    T acc = T(0);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const T p = r.v[6 * m] * s[0] + r.v[6 * m + 1] * s[1] + r.v[6 * m + 2] * s[2] + r.v[6 * m + 3] * s[3] +
                    r.v[6 * m + 4] * s[4] + r.v[6 * m + 5] * s[5];
        acc += p * p;
    }
    return acc;
}

__device__ __forceinline__ float log_t(float x) { return logf(x); }
__device__ __forceinline__ double log_t(double x) { return log(x); }

template <typename T, int MODE, bool RECOMP>
__global__ void __launch_bounds__(BLOCK_THREADS, (sizeof(T) == 4 ? 3 : 2)) k_sweep(SweepArgs<T> a, int colour) {
    constexpr bool ELASTIC = MODE == SWEEP_POINT || MODE == SWEEP_STRAIN;   // a point-zone elastic term
    constexpr bool STORED = ELASTIC && !RECOMP;                               // ... from the stored stress
    constexpr bool LIST = MODE == SWEEP_ZONE_LIST;
    const int r = __ldg(a.cta_rep + blockIdx.x);
    const Replica &R = a.reps[r];
    const int blk = (blockIdx.x - R.cta_off) * BLOCK_THREADS + threadIdx.x;  // block within the replica
    int nacc = 0;
    uint4 ent[4];   // zone mode: this thread's trials for the list
    int nent = 0;
    if (blk < R.nblk) {
        const int nbx = R.nbx, nby = R.nby, nbz = R.nbz;
        const int bx = blk % nbx, rr = blk / nbx;
        const int by = rr % nby, bz = rr / nby;
        const int sxy = nbx, sxz = nbx * nby;
        const int bxm = blk + (bx == 0 ? nbx - 1 : -1), bxp = blk + (bx == nbx - 1 ? 1 - nbx : 1);
        const int bym = blk + (by == 0 ? (nby - 1) * sxy : -sxy);
        const int byp = blk + (by == nby - 1 ? -(nby - 1) * sxy : sxy);
        const int bzm = blk + (bz == 0 ? (nbz - 1) * sxz : -sxz);
        const int bzp = blk + (bz == nbz - 1 ? -(nbz - 1) * sxz : sxz);
        uint4 *spins = a.spins + R.blk_off;
        const uint2 *q2 = reinterpret_cast<const uint2 *>(spins);
        const int oc = colour ^ 1;
        const uint4 own4 = spins[blk];
        const uint2 mine = colour ? make_uint2(own4.z, own4.w) : make_uint2(own4.x, own4.y);
        const uint2 O = oc ? make_uint2(own4.z, own4.w) : make_uint2(own4.x, own4.y);
        const uint2 Oxm = __ldg(q2 + 2 * bxm + oc), Oxp = __ldg(q2 + 2 * bxp + oc);
        const uint2 Oym = __ldg(q2 + 2 * bym + oc), Oyp = __ldg(q2 + 2 * byp + oc);
        const uint2 Ozm = __ldg(q2 + 2 * bzm + oc), Ozp = __ldg(q2 + 2 * bzp + oc);
        T sg[6][4];
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
        // the four sites' Philox draws first: four independent chains for the scheduler
        uint2 rnd[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int L = slot_local(4 * colour + i);
            const uint32_t x = 2u * bx + (L & 1), y = 2u * by + ((L >> 1) & 1), z = 2u * bz + (L >> 2);
            rnd[i] = philox_r01(x + (uint32_t)R.nx * (y + (uint32_t)R.ny * z), mcs, R.replica, 0u, R.key0, R.key1);
        }
        const T lam_sd_half = (T)R.lam_sd_half;
        // recompute mode: the cell's displacement gradients, formed at the first non-trivial trial
        CellGrad<T> g;
        T ebv[6];
        bool have_g = false;
        uint16_t out[4];
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
            T dHe = T(0);
            T er[6];   // recompute mode: the site's strain
            if (RECOMP && ELASTIC) {
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
                point_strain<T>(g, ebv, lx, ly, lz, er);
            }
            if (MODE == SWEEP_POINT) {
                T s[6];
                if (RECOMP) {
                    Row24<T> r;
                    r.load(a.ctab + 24ll * q);
                    hooke21<T>(r.v, er, s);
                } else {
#pragma unroll
                    for (int k = 0; k < 6; ++k) s[k] = sg[k][i];
                }
                dHe = lam_sd_half * (zone_phi<T>(a.wtab + 20ll * q, s) - zone_phi<T>(a.wtab + 20ll * qn, s));
            } else if (MODE == SWEEP_STRAIN) {
                // e held fixed (stored mode: e = S'(q) s): 1/2 (e.C'(q_new)e - e.C'(q)e)
                T e[6], sn[6], so[6];
                if (RECOMP) {
#pragma unroll
                    for (int k = 0; k < 6; ++k) e[k] = er[k];
                } else {
                    T s[6];
#pragma unroll
                    for (int k = 0; k < 6; ++k) s[k] = sg[k][i];
                    Row24<T> r;
                    r.load(a.stab + 24ll * q);
                    hooke21<T>(r.v, s, e);
                }
                {
                    Row24<T> r;
                    r.load(a.ctab + 24ll * qn);
                    hooke21<T>(r.v, e, sn);
                }
                {
                    Row24<T> r;
                    r.load(a.ctab + 24ll * q);
                    hooke21<T>(r.v, e, so);
                }
                T d = T(0);
#pragma unroll
                for (int k = 0; k < 6; ++k) d += e[k] * (sn[k] - so[k]);
                dHe = T(0.5) * (T)R.lam * d;
            }
            bool acc;
            if (!ELASTIC || dHe == T(0)) {
                acc = dE <= 0 || (unsigned long long)rn.y < __ldg(a.thr + dE);
            } else {
                const T H = a.J * (T)dE + dHe;
                const T u01 = ((T)rn.y + T(0.5)) * T(2.3283064365386963e-10);
                const T t = a.kT > T(0) ? -a.kT * log_t(u01) : T(0);
                acc = H <= t;
            }
            if (acc) {
                out[i] = qn;
                ++nacc;
            }
        }
        if (nacc) {
            uint2 w;
            w.x = (uint32_t)out[0] | ((uint32_t)out[1] << 16);
            w.y = (uint32_t)out[2] | ((uint32_t)out[3] << 16);
            reinterpret_cast<uint2 *>(spins)[2 * blk + colour] = w;
        }
    }
    if (LIST) {
        // warp-aggregated append: one atomic per warp, entries in lane order
        const int lane = threadIdx.x & 31;
        int incl = nent;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned base = 0;
        if (lane == 31 && total) base = atomicAdd(a.count, (unsigned)total);
        base = __shfl_sync(0xffffffffu, base, 31);
        const unsigned first = base + (unsigned)(incl - nent);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < nent) a.work[first + j] = ent[j];
        return;
    }
    // a CTA belongs to one replica: warp totals go to that replica's counter
    const unsigned tot = __reduce_add_sync(0xffffffffu, (unsigned)nacc);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&R.st->accepted, (unsigned long long)tot);
}

}  // namespace

template <typename T>
cudaError_t launch_sweep(const SweepArgs<T> &a, int colour, int mode, bool recompute, cudaStream_t s) {
    if (mode == SWEEP_POINT && recompute)
        k_sweep<T, SWEEP_POINT, true><<<a.nctas, BLOCK_THREADS, 0, s>>>(a, colour);
    else if (mode == SWEEP_POINT)
        k_sweep<T, SWEEP_POINT, false><<<a.nctas, BLOCK_THREADS, 0, s>>>(a, colour);
    else if (mode == SWEEP_STRAIN && recompute)
        k_sweep<T, SWEEP_STRAIN, true><<<a.nctas, BLOCK_THREADS, 0, s>>>(a, colour);
    else if (mode == SWEEP_STRAIN)
        k_sweep<T, SWEEP_STRAIN, false><<<a.nctas, BLOCK_THREADS, 0, s>>>(a, colour);
    else if (mode == SWEEP_ZONE_LIST)
        k_sweep<T, SWEEP_ZONE_LIST, false><<<a.nctas, BLOCK_THREADS, 0, s>>>(a, colour);
    else
        k_sweep<T, SWEEP_POTTS, false><<<a.nctas, BLOCK_THREADS, 0, s>>>(a, colour);
    return cudaGetLastError();
}

template cudaError_t launch_sweep<float>(const SweepArgs<float> &, int, int, bool, cudaStream_t);
template cudaError_t launch_sweep<double>(const SweepArgs<double> &, int, int, bool, cudaStream_t);

}  // namespace hmc
