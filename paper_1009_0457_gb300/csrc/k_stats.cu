// Stress of every material point (for the sweeps), the end-of-step reductions
// and loading control, statistics (unlike bonds, orientation volumes, texture
// bins) and the spin layout conversions.
#include "hmc_device.cuh"

namespace hmc {

namespace {

// Error-free sum of two floats (Knuth's TwoSum): a + b = s + e exactly.
struct FSum {
    float hi, lo;
    __device__ __forceinline__ void add(float x) {
        const float s = hi + x;
        const float bb = s - hi;
        const float e = (hi - (s - bb)) + (x - bb);
        hi = s;
        lo += e;
    }
    __device__ __forceinline__ void add(const FSum &o) {
        add(o.hi);
        lo += o.lo;
    }
};

// Per-thread accumulators of the seven reduced quantities.
template <typename T>
struct Acc7;
template <>
struct Acc7<float> {
    FSum v[7];
    __device__ __forceinline__ void zero() {
        for (int i = 0; i < 7; ++i) v[i].hi = v[i].lo = 0.f;
    }
    __device__ __forceinline__ void add(int i, float x) { v[i].add(x); }
    __device__ __forceinline__ void warp_reduce() {
#pragma unroll
        for (int off = 16; off; off >>= 1)
#pragma unroll
            for (int i = 0; i < 7; ++i) {
                FSum o;
                o.hi = __shfl_down_sync(0xffffffffu, v[i].hi, off);
                o.lo = __shfl_down_sync(0xffffffffu, v[i].lo, off);
                v[i].add(o);
            }
    }
    __device__ __forceinline__ double get(int i) const { return (double)v[i].hi + (double)v[i].lo; }
};
template <>
struct Acc7<double> {
    double v[7];
    __device__ __forceinline__ void zero() {
        for (int i = 0; i < 7; ++i) v[i] = 0.0;
    }
    __device__ __forceinline__ void add(int i, double x) { v[i] += x; }
    __device__ __forceinline__ void warp_reduce() {
#pragma unroll
        for (int off = 16; off; off >>= 1)
#pragma unroll
            for (int i = 0; i < 7; ++i) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
    }
    __device__ __forceinline__ double get(int i) const { return v[i]; }
};

// Stores of one colour's component of a block's stress: streaming (evict-first), so that the
// 403 MB written per pass do not push the spin field out of L2.  (Storing the red stress with
// the normal priority, for the red half sweep that reads it next, measured no faster.)
template <typename T>
__device__ __forceinline__ void store4(T *p, const T (&v)[4]);
template <>
__device__ __forceinline__ void store4<float>(float *p, const float (&v)[4]) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
}
template <>
__device__ __forceinline__ void store4<double>(double *p, const double (&v)[4]) {
    __stcs(reinterpret_cast<double2 *>(p), make_double2(v[0], v[1]));
    __stcs(reinterpret_cast<double2 *>(p) + 1, make_double2(v[2], v[3]));
}

// Stress of the eight points of each cell from the current displacement; the
// colour-packed stress array is what the half sweeps read.  Each CTA covers the
// 256 blocks of one replica's tile with STRESS_THREADS threads, each taking
// STRESS_CELLS blocks in turn (the warp reduction below is then paid once per
// STRESS_CELLS cells), and writes its partial sums of sigma and of 1/2 sigma.eps
// (a cell's eight points summed plainly, then FP32 TwoSum pairs or FP64 within a
// thread and a warp, by T, and FP64 across warps) for a fixed-order final
// reduction.
// threads of a stress CTA (measured on the 256^3 workload: 256 threads, one block each, 0.244 ms;
// 128 threads 0.180 ms; 64 threads 0.156 ms; 32 threads 0.156 ms).  Each thread loads its next
// block's corners and spins while it works on the current one (0.156 -> 0.150 ms), held to
// 128 registers in FP32 (eight CTAs per SM).
constexpr int STRESS_THREADS = 64;
constexpr int STRESS_CELLS = BLOCK_THREADS / STRESS_THREADS;
static_assert(BLOCK_THREADS % STRESS_THREADS == 0, "a tile splits evenly over the threads");

template <typename T, bool STORE>
__global__ void __launch_bounds__(STRESS_THREADS, sizeof(T) == 4 ? 8 : 1) k_stress(StressArgs<T> a) {
    __shared__ double red[STRESS_THREADS / 32][7];
    const int rep = __ldg(a.cta_rep + blockIdx.x);
    const Replica &R = a.reps[rep];
    const int t0 = (blockIdx.x - R.cta_off) * BLOCK_THREADS;
    Acc7<T> acc;
    acc.zero();
    T eb[6];
    load_ebar<T>(R.st, eb);
    const int nbx = R.nbx, nby = R.nby, nbz = R.nbz;
    const T *u = a.u + 3 * R.blk_off;
    T *sig = a.sig + 48ll * R.blk_off;
    // a cell's corner displacements and spins, loaded one cell ahead of its arithmetic
    auto load_cell = [&](int blk, T (&uc)[8][3], uint4 &sp) {
        const int bx = blk % nbx, rr = blk / nbx;
        const int by = rr % nby, bz = rr / nby;
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
        sp = __ldg(a.spins + R.blk_off + blk);
    };
    T un[8][3];
    uint4 spn = make_uint4(0, 0, 0, 0);
    int blk = t0 + threadIdx.x;
    if (blk < R.nblk) load_cell(blk, un, spn);
#pragma unroll 1
    for (int c8 = 0; c8 < STRESS_CELLS; ++c8) {
        if (blk >= R.nblk) break;
        T uc[8][3];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int d = 0; d < 3; ++d) uc[i][d] = un[i][d];
        const uint4 sp = spn;
        const int blk_next = blk + STRESS_THREADS;
        if (c8 + 1 < STRESS_CELLS && blk_next < R.nblk) load_cell(blk_next, un, spn);
        CellGrad<T> g;
        cell_gradients<T>(uc, g);
        T csum[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};   // this cell's eight points, plain sums
        Row24<T> row;
        uint32_t qprev = 0xffffffffu;
        // red slots 0..3, then black 4..7: each colour's stress is stored as soon as it is formed
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            T out[6][4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int slot = 4 * c + j, L = slot_local(slot);
                T e[6], st[6];
                point_strain<T>(g, eb, L & 1, (L >> 1) & 1, L >> 2, e);
                const uint32_t q = spin_of(sp, slot);  // points of a cell mostly share one orientation
                if (q != qprev) {
                    row.load(a.ctab + 24ll * q);
                    qprev = q;
                }
                hooke21<T>(row.v, e, st);
                T w = T(0);
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    out[k][j] = st[k];
                    csum[k] += st[k];
                    w += st[k] * e[k];
                }
                csum[6] += T(0.5) * w;
            }
            if (STORE) {
#pragma unroll
                for (int k = 0; k < 6; ++k) store4<T>(sig + 4ll * ((long long)(c * 6 + k) * R.nblk + blk), out[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < 7; ++k) acc.add(k, csum[k]);
        blk = blk_next;
    }
    acc.warp_reduce();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int i = 0; i < 7; ++i) red[warp][i] = acc.get(i);
    __syncthreads();
    if (threadIdx.x < 7) {
        double s = 0.0;
        for (int w = 0; w < STRESS_THREADS / 32; ++w) s += red[w][threadIdx.x];
        a.partials[7ll * blockIdx.x + threadIdx.x] = s;
    }
}

// End of a step: fixed-order FP64 reduction of each replica's stress partials,
// uniaxial control update of its mean strain, and its Monte Carlo step counter.
// GB300 retires few FP64 operations per SM, so the partials (one set of seven per
// stress CTA) are summed by END_GROUPS CTAs per replica: group g takes the CTAs
// g, g + END_GROUPS, ... (each thread in that order, then a tree over the threads),
// and the last group to arrive sums the group sums in group order and finishes.
__global__ void __launch_bounds__(256) k_end_mcs(const Replica *reps, double *partials, int nctas, int update_strain,
                                                  int advance) {
    __shared__ double red[256][7];
    __shared__ int last;
    const int r = blockIdx.x / END_GROUPS, grp = blockIdx.x % END_GROUPS;
    const Replica &R = reps[r];
    DevState *st = R.st;
    double *gsum = partials + 7ll * nctas + 7ll * END_GROUPS * r;   // this replica's group sums
    // the arrival counters follow the group sums of all replicas (gridDim.x = replicas x END_GROUPS)
    unsigned *arrive = reinterpret_cast<unsigned *>(partials + 7ll * nctas + 7ll * gridDim.x) + r;
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int p = grp + END_GROUPS * threadIdx.x; p < R.ncta; p += END_GROUPS * 256)
        for (int i = 0; i < 7; ++i) s[i] += partials[7ll * (R.cta_off + p) + i];
    for (int i = 0; i < 7; ++i) red[threadIdx.x][i] = s[i];
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w)
            for (int i = 0; i < 7; ++i) red[threadIdx.x][i] += red[threadIdx.x + w][i];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < 7; ++i) gsum[7 * grp + i] = red[0][i];
        __threadfence();
        last = atomicAdd(arrive, 1u) == END_GROUPS - 1;
    }
    __syncthreads();
    if (!last) return;
    // the last group of the replica: the group sums in group order
    __threadfence();
    if (threadIdx.x < 7) {
        double t = 0.0;
        for (int g = 0; g < END_GROUPS; ++g) t += __ldcg(gsum + 7 * g + threadIdx.x);
        red[0][threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double n_sites = 8.0 * (double)R.nblk;
        double mean[6];
        int bad = 0;
        for (int i = 0; i < 6; ++i) {
            mean[i] = red[0][i] / n_sites;
            st->mean_sigma[i] = mean[i];
            bad |= !isfinite(mean[i]);
        }
        st->energy = red[0][6];
        bad |= !isfinite(red[0][6]);
        if (bad) st->nonfinite = 1;
        if (update_strain && st->bc == 0 && !bad) {
            // remove the lateral mean stress with the Reuss compliance, then restore
            // the axial strain along the uniaxial-stress direction S_R (n(x)n)
            double nsn = 0.0;
            for (int i = 0; i < 6; ++i) nsn += st->axNs[i] * mean[i];
            double r[6], e[6];
            for (int i = 0; i < 6; ++i) r[i] = mean[i] - nsn * st->axN[i];
            for (int i = 0; i < 6; ++i) {
                double d = 0.0;
                for (int j = 0; j < 6; ++j) d += st->sr[6 * i + j] * r[j];
                e[i] = st->ebar[i] - d;
            }
            double ne = 0.0;
            for (int i = 0; i < 6; ++i) ne += st->axN[i] * e[i];
            const double beta = (st->eps0 - ne) / st->axNB;
            for (int i = 0; i < 6; ++i) {
                st->ebar[i] = e[i] + beta * st->axB[i];
                st->ebar_f[i] = (float)st->ebar[i];
            }
        }
        if (update_strain && st->bc == 2 && !bad) {
            // stress control: Ebar += S_R (sig0 n(x)n - <sigma>)
            double e[6];
            for (int i = 0; i < 6; ++i) {
                double d = 0.0;
                for (int j = 0; j < 6; ++j) d += st->sr[6 * i + j] * (st->sig0 * st->axN[j] - mean[j]);
                e[i] = st->ebar[i] + d;
            }
            for (int i = 0; i < 6; ++i) {
                st->ebar[i] = e[i];
                st->ebar_f[i] = (float)e[i];
            }
        }
        if (advance) st->mcs += 1;
        *arrive = 0u;   // ready for the next launch
    }
}

// Upload check: flag any orientation index >= Q (8 indices per thread, 16 B loads).
__global__ void k_check_spins(const uint16_t *__restrict__ nat, long long n, int nq, DevState *st) {
    const long long n8 = n >> 3;
    int bad = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += (long long)gridDim.x * blockDim.x) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(nat) + i);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) bad |= ((w[k] & 0xffffu) >= (uint32_t)nq) | ((w[k] >> 16) >= (uint32_t)nq);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->bad_spin, 1);
}

// natural uint16 field <-> 2x2x2 blocks in slot order
__global__ void k_pack_spins(const uint16_t *__restrict__ nat, uint4 *__restrict__ blk, int nx, int ny, int nz) {
    const int nbx = nx >> 1, nby = ny >> 1, nbz = nz >> 1;
    const long long nblk = (long long)nbx * nby * nbz;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += (long long)gridDim.x * blockDim.x) {
        const int bx = (int)(b % nbx);
        const long long r = b / nbx;
        const int by = (int)(r % nby), bz = (int)(r / nby);
        uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int L = slot_local(s);
            const long long x = 2 * bx + (L & 1), y = 2 * by + ((L >> 1) & 1), z = 2 * bz + (L >> 2);
            const uint32_t q = nat[x + nx * (y + (long long)ny * z)];
            w[s >> 1] |= (s & 1) ? (q << 16) : q;
        }
        blk[b] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

__global__ void k_unpack_spins(const uint4 *__restrict__ blk, uint16_t *__restrict__ nat, int nx, int ny, int nz) {
    const int nbx = nx >> 1, nby = ny >> 1, nbz = nz >> 1;
    const long long nblk = (long long)nbx * nby * nbz;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += (long long)gridDim.x * blockDim.x) {
        const int bx = (int)(b % nbx);
        const long long r = b / nbx;
        const int by = (int)(r % nby), bz = (int)(r / nby);
        const uint4 v = blk[b];
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int L = slot_local(s);
            const long long x = 2 * bx + (L & 1), y = 2 * by + ((L >> 1) & 1), z = 2 * bz + (L >> 2);
            nat[x + nx * (y + (long long)ny * z)] = spin_of(v, s);
        }
    }
}

// Unlike +x/+y/+z bonds of every site (each bond once) and the volume of
// every orientation, one thread per block.
__global__ void __launch_bounds__(256) k_bonds_counts(const uint4 *__restrict__ spins, int nbx, int nby, int nbz,
                                                      int nq, int smem_bins, unsigned long long *counts,
                                                      DevState *st) {
    extern __shared__ unsigned int hist[];
    if (smem_bins)
        for (int i = threadIdx.x; i < nq; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const long long nblk = (long long)nbx * nby * nbz;
    unsigned long long unlike = 0;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += (long long)gridDim.x * blockDim.x) {
        const int bx = (int)(b % nbx);
        const long long r = b / nbx;
        const int by = (int)(r % nby), bz = (int)(r / nby);
        const uint4 me = __ldg(spins + b);
        const uint4 px = __ldg(spins + (b + (bx == nbx - 1 ? 1 - nbx : 1)));
        const uint4 py = __ldg(spins + (b + (by == nby - 1 ? -(long long)(nby - 1) * nbx : nbx)));
        const uint4 pz = __ldg(spins + (b + (bz == nbz - 1 ? -(long long)(nbz - 1) * nbx * nby : (long long)nbx * nby)));
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int L = slot_local(s);
            const int lx = L & 1, ly = (L >> 1) & 1, lz = L >> 2;
            const uint16_t q = spin_of(me, s);
            const uint16_t qx = lx ? spin_of(px, local_slot(L ^ 1)) : spin_of(me, local_slot(L ^ 1));
            const uint16_t qy = ly ? spin_of(py, local_slot(L ^ 2)) : spin_of(me, local_slot(L ^ 2));
            const uint16_t qz = lz ? spin_of(pz, local_slot(L ^ 4)) : spin_of(me, local_slot(L ^ 4));
            unlike += (q != qx) + (q != qy) + (q != qz);
            if (smem_bins)
                atomicAdd(&hist[q], 1u);
            else
                atomicAdd(&counts[q], 1ull);
        }
    }
    for (int off = 16; off; off >>= 1) unlike += __shfl_down_sync(0xffffffffu, unlike, off);
    if ((threadIdx.x & 31) == 0 && unlike) atomicAdd(&st->unlike, unlike);
    __syncthreads();
    if (smem_bins)
        for (int i = threadIdx.x; i < nq; i += blockDim.x)
            if (hist[i]) atomicAdd(&counts[i], (unsigned long long)hist[i]);
}

__global__ void k_bins(const unsigned long long *counts, const int32_t *binmap, int nq, int nbins,
                       unsigned long long *bins, double *fractions, long long n_sites) {
    for (int q = threadIdx.x; q < nq; q += blockDim.x) atomicAdd(&bins[binmap[q]], counts[q]);
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) fractions[b] = (double)bins[b] / (double)n_sites;
}

}  // namespace

template <typename T>
cudaError_t launch_stress(const StressArgs<T> &a, bool store, cudaStream_t s) {
    if (store)
        k_stress<T, true><<<a.nctas, STRESS_THREADS, 0, s>>>(a);
    else
        k_stress<T, false><<<a.nctas, STRESS_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}
template cudaError_t launch_stress<float>(const StressArgs<float> &, bool, cudaStream_t);
template cudaError_t launch_stress<double>(const StressArgs<double> &, bool, cudaStream_t);

cudaError_t launch_end_mcs(const Replica *reps, int nrep, double *partials, int nctas, int update_strain, int advance,
                           cudaStream_t s) {
    k_end_mcs<<<nrep * END_GROUPS, 256, 0, s>>>(reps, partials, nctas, update_strain, advance);
    return cudaGetLastError();
}

static int grid_for(long long n) {
    long long g = (n + 255) / 256;
    if (g > 65535ll * 8) g = 65535ll * 8;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t launch_check_spins(const uint16_t *nat, long long n, int nq, DevState *st, cudaStream_t s) {
    k_check_spins<<<grid_for(n >> 3), 256, 0, s>>>(nat, n, nq, st);
    return cudaGetLastError();
}

cudaError_t launch_pack_spins(const uint16_t *nat, uint4 *blk, int nx, int ny, int nz, cudaStream_t s) {
    const long long nblk = (long long)(nx / 2) * (ny / 2) * (nz / 2);
    k_pack_spins<<<grid_for(nblk), 256, 0, s>>>(nat, blk, nx, ny, nz);
    return cudaGetLastError();
}

cudaError_t launch_unpack_spins(const uint4 *blk, uint16_t *nat, int nx, int ny, int nz, cudaStream_t s) {
    const long long nblk = (long long)(nx / 2) * (ny / 2) * (nz / 2);
    k_unpack_spins<<<grid_for(nblk), 256, 0, s>>>(blk, nat, nx, ny, nz);
    return cudaGetLastError();
}

cudaError_t launch_bonds_counts(const uint4 *blk, int nbx, int nby, int nbz, int nq, unsigned long long *counts,
                                DevState *st, cudaStream_t s) {
    const long long nblk = (long long)nbx * nby * nbz;
    const int smem_bins = nq <= 12288;
    long long g = (nblk + 255) / 256;
    if (g > 4096) g = 4096;  // grid-stride: fewer, longer CTAs amortise the shared histogram flush
    k_bonds_counts<<<(int)g, 256, smem_bins ? nq * sizeof(unsigned int) : 0, s>>>(blk, nbx, nby, nbz, nq, smem_bins,
                                                                                counts, st);
    return cudaGetLastError();
}

cudaError_t launch_bins(const unsigned long long *counts, const int32_t *binmap, int nq, int nbins,
                        unsigned long long *bins, double *fractions, long long n_sites, cudaStream_t s) {
    k_bins<<<1, 1024, 0, s>>>(counts, binmap, nq, nbins, bins, fractions, n_sites);
    return cudaGetLastError();
}

}  // namespace hmc
