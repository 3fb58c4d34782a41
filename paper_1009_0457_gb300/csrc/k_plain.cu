// The explicit MPM step in its plain, unfused, incremental FP64 form (Sec. "Elastic
// Deformation": nodal velocity -> particle velocity gradient -> strain increment ->
// Hooke's law applied to update the particle stresses -> internal nodal forces),
// kept as the baseline that the fused total-form step is measured against.
//
// Each step is three kernels over state in global memory:
//   k_plain_p2g   per cell: internal forces of its eight points on its eight corners,
//                 f_I -= V sigma_p . grad N_I(x_p), every point and corner in turn
//   k_plain_grid  per node: the sum of its eight cells' corner forces, then the damped
//                 update v <- (1 - zeta) v + dt f / m, u <- u + dt v
//   k_plain_g2p   per cell: the strain increment of each point from its corners'
//                 displacement increments dt v, and sigma_p <- sigma_p + C'(q_p) d eps
// with the point stresses (6 per point) and the cell forces (24 per cell) stored between
// them.  The stresses start each call from the total form sigma = C'(q)(Ebar + B u).
// While the spins are fixed the result equals the fused step's to rounding.
#include "hmc_device.cuh"

namespace hmc {

namespace {

// gradient of the trilinear shape function of corner (I,J,K) at point (a,b,c) of a cell
// (coordinates 1/4 and 3/4 of the edge h = 2 voxels; the 1/h is in the +-1/2 factors)
__device__ __forceinline__ void plain_grad(int a, int b, int c, int I, int J, int K, double (&g)[3]) {
    const double xa = a ? 0.75 : 0.25, xb = b ? 0.75 : 0.25, xc = c ? 0.75 : 0.25;
    const double Na = I ? xa : 1.0 - xa, Nb = J ? xb : 1.0 - xb, Nc = K ? xc : 1.0 - xc;
    g[0] = (I ? 0.5 : -0.5) * Nb * Nc;
    g[1] = Na * (J ? 0.5 : -0.5) * Nc;
    g[2] = Na * Nb * (K ? 0.5 : -0.5);
}

// the cell's corner node indices (periodic)
__device__ __forceinline__ void cell_corners(const PlainArgs &a, int blk, int (&n)[8]) {
    const int bx = blk % a.nbx, r = blk / a.nbx, by = r % a.nby, bz = r / a.nby;
#pragma unroll
    for (int K = 0; K < 2; ++K)
#pragma unroll
        for (int J = 0; J < 2; ++J)
#pragma unroll
            for (int I = 0; I < 2; ++I) {
                const int gi = bx + I == a.nbx ? 0 : bx + I, gj = by + J == a.nby ? 0 : by + J;
                const int gk = bz + K == a.nbz ? 0 : bz + K;
                n[corner(I, J, K)] = gi + a.nbx * (gj + a.nby * gk);
            }
}

// sigma = C'(q)(Ebar + B u) at every point: the starting stress of the incremental steps
__global__ void __launch_bounds__(128) k_plain_init(PlainArgs a) {
    const int blk = blockIdx.x * blockDim.x + threadIdx.x;
    if (blk >= a.nblk) return;
    int n[8];
    cell_corners(a, blk, n);
    double uc[8][3];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int d = 0; d < 3; ++d) uc[i][d] = a.u[3 * n[i] + d];
    CellGrad<double> g;
    cell_gradients<double>(uc, g);
    const uint4 sp = a.spins[blk];
    double eb[6];
    load_ebar<double>(a.st, eb);
#pragma unroll
    for (int L = 0; L < 8; ++L) {
        double e[6], s[6];
        point_strain<double>(g, eb, L & 1, (L >> 1) & 1, L >> 2, e);
        Row24<double> row;
        row.load(a.ctab + 24ll * spin_of(sp, local_slot(L)));
        hooke21<double>(row.v, e, s);
#pragma unroll
        for (int k = 0; k < 6; ++k) a.sig[((long long)k * a.nblk + blk) * 8 + L] = s[k];
    }
}

__global__ void __launch_bounds__(128) k_plain_p2g(PlainArgs a) {
    const int blk = blockIdx.x * blockDim.x + threadIdx.x;
    if (blk >= a.nblk) return;
    double f[8][3];
#pragma unroll
    for (int i = 0; i < 8; ++i) f[i][0] = f[i][1] = f[i][2] = 0.0;
    for (int L = 0; L < 8; ++L) {
        double s[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) s[k] = a.sig[((long long)k * a.nblk + blk) * 8 + L];
#pragma unroll
        for (int cr = 0; cr < 8; ++cr) {
            double g[3];
            plain_grad(L & 1, (L >> 1) & 1, L >> 2, cr & 1, (cr >> 1) & 1, cr >> 2, g);
            // f -= V sigma . grad N, V = 1 voxel; sigma in Voigt order xx yy zz yz xz xy
            f[cr][0] -= s[0] * g[0] + s[5] * g[1] + s[4] * g[2];
            f[cr][1] -= s[5] * g[0] + s[1] * g[1] + s[3] * g[2];
            f[cr][2] -= s[4] * g[0] + s[3] * g[1] + s[2] * g[2];
        }
    }
#pragma unroll
    for (int cr = 0; cr < 8; ++cr)
#pragma unroll
        for (int d = 0; d < 3; ++d) a.fcell[(long long)(3 * cr + d) * a.nblk + blk] = f[cr][d];
}

__global__ void __launch_bounds__(128) k_plain_grid(PlainArgs a) {
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= a.nblk) return;
    const int i = node % a.nbx, r = node / a.nbx, j = r % a.nby, k = r / a.nby;
    double F[3] = {0.0, 0.0, 0.0};
    // the node is corner (I,J,K) of the cell whose lower corner is (i-I, j-J, k-K)
#pragma unroll
    for (int K = 0; K < 2; ++K)
#pragma unroll
        for (int J = 0; J < 2; ++J)
#pragma unroll
            for (int I = 0; I < 2; ++I) {
                const int ci = i - I < 0 ? a.nbx - 1 : i - I, cj = j - J < 0 ? a.nby - 1 : j - J;
                const int ck = k - K < 0 ? a.nbz - 1 : k - K;
                const long long cell = ci + (long long)a.nbx * (cj + (long long)a.nby * ck);
#pragma unroll
                for (int d = 0; d < 3; ++d) F[d] += a.fcell[(long long)(3 * corner(I, J, K) + d) * a.nblk + cell];
            }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double v = a.keep * a.v[3 * node + d] + a.dt_over_m * F[d];
        a.v[3 * node + d] = v;
        a.u_out[3 * node + d] = a.u[3 * node + d] + a.dt * v;
    }
}

__global__ void __launch_bounds__(128) k_plain_g2p(PlainArgs a) {
    const int blk = blockIdx.x * blockDim.x + threadIdx.x;
    if (blk >= a.nblk) return;
    int n[8];
    cell_corners(a, blk, n);
    double du[8][3];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int d = 0; d < 3; ++d) du[i][d] = a.dt * a.v[3 * n[i] + d];
    const uint4 sp = a.spins[blk];
    for (int L = 0; L < 8; ++L) {
        // velocity gradient times dt at the point: G[d][x] = sum_corners du_d dN/dx
        double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int cr = 0; cr < 8; ++cr) {
            double g[3];
            plain_grad(L & 1, (L >> 1) & 1, L >> 2, cr & 1, (cr >> 1) & 1, cr >> 2, g);
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
                for (int x = 0; x < 3; ++x) G[d][x] += du[cr][d] * g[x];
        }
        const double de[6] = {G[0][0], G[1][1], G[2][2], G[1][2] + G[2][1], G[0][2] + G[2][0], G[0][1] + G[1][0]};
        Row24<double> row;
        row.load(a.ctab + 24ll * spin_of(sp, local_slot(L)));
        double ds[6];
        hooke21<double>(row.v, de, ds);
#pragma unroll
        for (int k = 0; k < 6; ++k) a.sig[((long long)k * a.nblk + blk) * 8 + L] += ds[k];
    }
}

}  // namespace

cudaError_t launch_plain_init(const PlainArgs &a, cudaStream_t s) {
    k_plain_init<<<(a.nblk + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

// one plain step: forces from the current point stresses, the node update into u_out, and
// the stress increment from the nodes' new velocities
cudaError_t launch_plain_step(const PlainArgs &a, cudaStream_t s) {
    const int grid = (a.nblk + 127) / 128;
    k_plain_p2g<<<grid, 128, 0, s>>>(a);
    k_plain_grid<<<grid, 128, 0, s>>>(a);
    k_plain_g2p<<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace hmc
