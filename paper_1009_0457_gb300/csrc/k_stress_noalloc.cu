// Allocation-free stress pass: hmc_stress_noalloc (declared in include/hmc.h).
//
// Some callers cannot allocate device memory at the point where they need the
// stress field: code running inside another framework's memory pool or a
// fixed-budget arena, or code that may not call cudaMalloc/cudaFree at that
// point because those calls synchronise the device.  For them this entry point
// computes the same quantities as hmc_compute_stress + hmc_get_stress
// (FP32 stress of every point, FP64 mean stress and elastic energy) from
// caller-owned device buffers, and keeps its only scratch -- the per-CTA
// partial sums of the fixed-order reduction -- in a file-scope device array.
//
// Limits and sharing: the array holds NOALLOC_MAX_CTAS partial-sum slots of
// 8 doubles (512 KiB, resident on every GPU that loads the library until the
// process exits); one CTA covers 256 cells of 2x2x2 points, so grids of up to
// 2,097,152 cells (16,777,216 points) are served -- 256^3 is the largest cube
// accepted -- and larger ones are rejected.  Every call uses the same array and
// leaves its partial sums there; each call overwrites every slot it reads, so
// nothing has to start at zero, but two calls whose work overlaps on the GPU
// (different streams, no ordering) race on the array.  The array's device
// address is looked up once per device and kept for the life of the process,
// which assumes the device's primary context and no cudaDeviceReset after the
// first call.
#include <cmath>
#include <mutex>
#include <string>

#include "hmc.h"
#include "hmc_device.cuh"

namespace hmc {
void set_unbound_error(const std::string &msg);  // message for hmc_last_error(NULL)
}

namespace {

constexpr int NOALLOC_MAX_CTAS = 8192;
constexpr int NOALLOC_THREADS = 256;

static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_CTAS * 8];

struct NoallocArgs {
    const uint16_t *spins;  // natural order
    const float *u;         // nnodes x 3
    const float *ctab;      // Q x 36, full Voigt C'(q), row-major
    float *sigma;           // N x 6, natural order
    double *partials;       // device address of g_noalloc_partials
    double *mean;           // 6
    double *energy;         // 1
    float eb[6];
    int nx, ny, nz, nbx, nby, nbz;
    long long nblk, n_sites;
};

__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float x) {
    const float s = hi + x;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
}

// One thread per 2x2x2 cell: strain of its eight points from the trilinear
// nodal field, Hooke's law with the point's rotated stiffness, natural-order
// stress out, and per-CTA FP64 partial sums of sigma and 1/2 sigma.eps.
__global__ void __launch_bounds__(NOALLOC_THREADS) k_stress_noalloc(NoallocArgs a) {
    __shared__ double red[NOALLOC_THREADS / 32][7];
    float hi[7], lo[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) hi[i] = lo[i] = 0.f;
    const long long blk = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (blk < a.nblk) {
        const int bx = (int)(blk % a.nbx);
        const long long r = blk / a.nbx;
        const int by = (int)(r % a.nby), bz = (int)(r / a.nby);
        float u[8][3];
#pragma unroll
        for (int K = 0; K < 2; ++K)
#pragma unroll
            for (int J = 0; J < 2; ++J)
#pragma unroll
                for (int I = 0; I < 2; ++I) {
                    const int gi = bx + I == a.nbx ? 0 : bx + I;
                    const int gj = by + J == a.nby ? 0 : by + J;
                    const int gk = bz + K == a.nbz ? 0 : bz + K;
                    const long long n = 3ll * (gi + (long long)a.nbx * (gj + (long long)a.nby * gk));
#pragma unroll
                    for (int d = 0; d < 3; ++d) u[hmc::corner(I, J, K)][d] = __ldg(a.u + n + d);
                }
        hmc::CellGrad<float> g;
        hmc::cell_gradients<float>(u, g);
#pragma unroll
        for (int L = 0; L < 8; ++L) {
            const int lx = L & 1, ly = (L >> 1) & 1, lz = L >> 2;
            const long long x = 2 * bx + lx, y = 2 * by + ly, z = 2 * bz + lz;
            const long long p = x + a.nx * (y + (long long)a.ny * z);
            float e[6], s[6];
            hmc::point_strain<float>(g, a.eb, lx, ly, lz, e);
            const float *c = a.ctab + 36ll * __ldg(a.spins + p);
            float w = 0.f;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < 6; ++j) acc += __ldg(c + 6 * i + j) * e[j];
                s[i] = acc;
                w += acc * e[i];
                two_sum_add(hi[i], lo[i], acc);
            }
            two_sum_add(hi[6], lo[6], 0.5f * w);
#pragma unroll
            for (int i = 0; i < 6; ++i) a.sigma[6 * p + i] = s[i];
        }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1)
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            const float oh = __shfl_down_sync(0xffffffffu, hi[i], off);
            const float ol = __shfl_down_sync(0xffffffffu, lo[i], off);
            two_sum_add(hi[i], lo[i], oh);
            lo[i] += ol;
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int i = 0; i < 7; ++i) red[warp][i] = (double)hi[i] + (double)lo[i];
    __syncthreads();
    if (threadIdx.x < 7) {
        double s = 0.0;
        for (int w = 0; w < NOALLOC_THREADS / 32; ++w) s += red[w][threadIdx.x];
        a.partials[8ll * blockIdx.x + threadIdx.x] = s;  // every slot this call reads is written here
    }
}

// Fixed-order FP64 sum of the partials of all CTAs.
__global__ void __launch_bounds__(256) k_noalloc_finish(NoallocArgs a, int nparts) {
    __shared__ double red[256][7];
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int p = threadIdx.x; p < nparts; p += 256)
        for (int i = 0; i < 7; ++i) s[i] += a.partials[8ll * p + i];
    for (int i = 0; i < 7; ++i) red[threadIdx.x][i] = s[i];
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w)
            for (int i = 0; i < 7; ++i) red[threadIdx.x][i] += red[threadIdx.x + w][i];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < 6; ++i) a.mean[i] = red[0][i] / (double)a.n_sites;
        *a.energy = red[0][6];
    }
}

// Device address of the scratch array, looked up once per device.
std::mutex g_setup_mutex;
double *g_partials_addr[64] = {nullptr};

}  // namespace

extern "C" hmc_status hmc_stress_noalloc(const uint16_t *d_spins, const float *d_u, const float *d_ctab,
                                         const double *strain_bar, int32_t nx, int32_t ny, int32_t nz,
                                         float *d_sigma, double *d_mean, double *d_energy, void *stream) {
    if (!d_spins || !d_u || !d_ctab || !strain_bar || !d_sigma || !d_mean || !d_energy) {
        hmc::set_unbound_error("hmc_stress_noalloc: NULL pointer argument");
        return HMC_ERR_ARG;
    }
    if (nx < 4 || ny < 4 || nz < 4 || nx % 2 || ny % 2 || nz % 2) {
        hmc::set_unbound_error("hmc_stress_noalloc: grid edges must be even and >= 4");
        return HMC_ERR_ARG;
    }
    const long long nblk = (long long)(nx / 2) * (ny / 2) * (nz / 2);
    const long long nparts = (nblk + NOALLOC_THREADS - 1) / NOALLOC_THREADS;
    if (nparts > NOALLOC_MAX_CTAS) {
        hmc::set_unbound_error("hmc_stress_noalloc: " + std::to_string(8 * nblk) +
                               " points exceed the limit of " +
                               std::to_string(8ll * NOALLOC_THREADS * NOALLOC_MAX_CTAS) +
                               " points of its fixed scratch array");
        return HMC_ERR_ARG;
    }
    for (int i = 0; i < 6; ++i)
        if (!std::isfinite(strain_bar[i])) {
            hmc::set_unbound_error("hmc_stress_noalloc: non-finite strain_bar");
            return HMC_ERR_ARG;
        }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        hmc::set_unbound_error(std::string("hmc_stress_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return HMC_ERR_CUDA;
    }
    double *partials = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partials_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess) {
                hmc::set_unbound_error(std::string("hmc_stress_noalloc: cudaGetSymbolAddress: ") +
                                       cudaGetErrorString(e));
                return HMC_ERR_CUDA;
            }
            g_partials_addr[dev] = static_cast<double *>(p);
        }
        partials = g_partials_addr[dev];
    }
    NoallocArgs a;
    a.spins = d_spins;
    a.u = d_u;
    a.ctab = d_ctab;
    a.sigma = d_sigma;
    a.partials = partials;
    a.mean = d_mean;
    a.energy = d_energy;
    for (int i = 0; i < 6; ++i) a.eb[i] = (float)strain_bar[i];
    a.nx = nx; a.ny = ny; a.nz = nz;
    a.nbx = nx / 2; a.nby = ny / 2; a.nbz = nz / 2;
    a.nblk = nblk;
    a.n_sites = 8 * nblk;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_stress_noalloc<<<(unsigned)nparts, NOALLOC_THREADS, 0, s>>>(a);
    k_noalloc_finish<<<1, 256, 0, s>>>(a, (int)nparts);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        hmc::set_unbound_error(std::string("hmc_stress_noalloc: launch: ") + cudaGetErrorString(e));
        return HMC_ERR_CUDA;
    }
    return HMC_OK;
}
