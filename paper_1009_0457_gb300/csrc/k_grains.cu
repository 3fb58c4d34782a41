// Grain count of one replica: grains are the face-connected sets of sites of
// one orientation on the periodic lattice (a grain's volume is the number of
// sites it holds, Sec. "Microstructural Evolution"; the mean grain volume is the
// site count over the grain count).  Union-find over the sites with labels in
// block-slot order (8 block + slot): every union hooks the larger root under the
// smaller one with one compare-and-swap, so a parent is always smaller than its
// child and the forest stays acyclic under any interleaving; finds halve paths
// (writing an ancestor is always a valid parent).  The count is the number of
// roots, independent of the order in which the unions ran.  Every loop is capped;
// a capped-out loop sets the error word instead of spinning.
#include <algorithm>

#include "hmc_device.cuh"

namespace hmc {

namespace {

constexpr int CC_CAP = 1 << 22;

__device__ __forceinline__ unsigned cc_load(const unsigned *p) { return *reinterpret_cast<const volatile unsigned *>(p); }

__device__ __forceinline__ unsigned cc_find(unsigned *parent, unsigned x, int *err) {
    for (int it = 0; it < CC_CAP; ++it) {
        const unsigned p = cc_load(parent + x);
        if (p == x) return x;
        const unsigned gp = cc_load(parent + p);
        if (gp != p) parent[x] = gp;
        x = gp;
    }
    *err = 1;
    return x;
}

__device__ __forceinline__ void cc_unite(unsigned *parent, unsigned a, unsigned b, int *err) {
    for (int it = 0; it < CC_CAP; ++it) {
        a = cc_find(parent, a, err);
        b = cc_find(parent, b, err);
        if (a == b) return;
        const unsigned lo = min(a, b), hi = max(a, b);
        if (atomicCAS(parent + hi, hi, lo) == hi) return;
    }
    *err = 1;
}

__global__ void k_cc_init(unsigned *parent, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        parent[i] = (unsigned)i;
}

// one thread per 2x2x2 block: its eight sites against their +x, +y, +z neighbours
__global__ void k_cc_union(const uint4 *__restrict__ spins, int nbx, int nby, int nbz, unsigned *parent, int *err) {
    const long long nblk = (long long)nbx * nby * nbz;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += (long long)gridDim.x * blockDim.x) {
        const int bx = (int)(b % nbx);
        const long long r = b / nbx;
        const int by = (int)(r % nby), bz = (int)(r / nby);
        const long long bxp = b + (bx == nbx - 1 ? 1 - nbx : 1);
        const long long byp = b + (by == nby - 1 ? -(long long)(nby - 1) * nbx : nbx);
        const long long bzp = b + (bz == nbz - 1 ? -(long long)(nbz - 1) * nbx * nby : (long long)nbx * nby);
        const uint4 me = __ldg(spins + b), px = __ldg(spins + bxp), py = __ldg(spins + byp), pz = __ldg(spins + bzp);
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int L = slot_local(s);
            const int lx = L & 1, ly = (L >> 1) & 1, lz = L >> 2;
            const unsigned id = (unsigned)(8 * b + s);
            const uint16_t q = spin_of(me, s);
            const int sx = local_slot(L ^ 1), sy = local_slot(L ^ 2), sz = local_slot(L ^ 4);
            if (q == (lx ? spin_of(px, sx) : spin_of(me, sx)))
                cc_unite(parent, id, (unsigned)(8 * (lx ? bxp : b) + sx), err);
            if (q == (ly ? spin_of(py, sy) : spin_of(me, sy)))
                cc_unite(parent, id, (unsigned)(8 * (ly ? byp : b) + sy), err);
            if (q == (lz ? spin_of(pz, sz) : spin_of(me, sz)))
                cc_unite(parent, id, (unsigned)(8 * (lz ? bzp : b) + sz), err);
        }
    }
}

__global__ void k_cc_roots(const unsigned *parent, long long n, unsigned long long *count) {
    unsigned long long c = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        c += parent[i] == (unsigned)i;
    for (int off = 16; off; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

}  // namespace

cudaError_t launch_grain_count(const uint4 *spins, int nbx, int nby, int nbz, unsigned *parent,
                               unsigned long long *count, int *err, cudaStream_t s) {
    const long long nblk = (long long)nbx * nby * nbz, n = 8 * nblk;
    const int g1 = (int)std::min<long long>((n + 255) / 256, 8192), g2 = (int)std::min<long long>((nblk + 255) / 256, 8192);
    cudaError_t e;
    if ((e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(err, 0, sizeof(int), s)) != cudaSuccess) return e;
    k_cc_init<<<g1, 256, 0, s>>>(parent, n);
    k_cc_union<<<g2, 256, 0, s>>>(spins, nbx, nby, nbz, parent, err);
    k_cc_roots<<<g1, 256, 0, s>>>(parent, n, count);
    return cudaGetLastError();
}

}  // namespace hmc
