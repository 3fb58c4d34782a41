// Fused explicit MPM step (Sec. "Elastic Deformation"): for every material
// point strain from the nodal displacement, Hooke's law (Eq. 1) with the
// point's rotated stiffness, internal nodal force, then the damped
// velocity / displacement update of every node -- one kernel, one pass over
// the spins and the nodal state.
//
// Tiling: a CTA of 16x16 threads computes a 16x16 patch of cells per cell
// plane (one thread per cell, all eight points of the cell) and owns the
// 15x15 nodes whose four lower and four upper cells all lie in the patch.  It
// marches up a chunk of planes in z: each cell writes its eight nodal force
// contributions to shared memory, and a node's force is the sum of its four
// cells below (carried in registers from the previous plane) and four above.
// Node planes are triple-buffered in shared memory (structure of arrays, so
// neighbouring threads hit neighbouring banks) and the next plane's spins and
// the owned node's velocity are fetched one plane ahead.  Displacements are
// read from one buffer and written to the other, so CTAs never race on the halo.
//
// Scheduling: the (tile, plane) space is cut into one contiguous range per
// resident CTA (a persistent grid of occupancy x SMs), so every CTA marches
// about the same number of planes and pays the one-plane restart only where
// its range enters a new tile.
//
// Scaling: the interpolation weights 3/4 and 1/4 of the trilinear shape
// functions at the points 1/4 and 3/4 of the cell are applied as 3 and 1; the
// factors 1/16 and 1/h are folded into the displacements held in shared memory
// (u/32) and into the force constant of the node update (-dt/(32 m)) -- both
// exact powers of two.
#include "hmc_device.cuh"

namespace hmc {

namespace {

constexpr int CT = 16;        // cells per patch edge = threads per edge
constexpr int OT = CT - 1;    // owned nodes per patch edge
constexpr int NT = CT + 1;    // node-plane tile edge (one node of halo each side)
constexpr int NTHR = CT * CT;

template <typename T>
struct MpmSmem {
    T us[3][3][NT][NT];   // node planes (buffer, component, j, i)
    T fb[4][3][CT][CT];   // cell contributions to their lower corner nodes (corner I+2J, component)
    T ft[4][3][CT][CT];   // ... to their upper corner nodes
};

template <typename T>
__device__ __forceinline__ void load_plane(MpmSmem<T> &sm, int buf, const T *__restrict__ u, int i0, int j0, int k,
                                           int nbx, int nby, int nbz) {
    const int gk = wrapi(k, nbz);
    for (int t = threadIdx.x; t < NT * NT; t += NTHR) {
        const int li = t % NT, lj = t / NT;
        const int gi = wrapi(i0 - 1 + li, nbx), gj = wrapi(j0 - 1 + lj, nby);
        const long long n = 3ll * (gi + (long long)nbx * (gj + (long long)nby * gk));
        sm.us[buf][0][lj][li] = __ldg(u + n) * T(0.03125);
        sm.us[buf][1][lj][li] = __ldg(u + n + 1) * T(0.03125);
        sm.us[buf][2][lj][li] = __ldg(u + n + 2) * T(0.03125);
    }
}

// 2x2 -> 2x2 transform with weights 3 (same side) and 1 (other side) in both
// indices: o[b][c] = sum_J sum_K W(J,b) W(K,c) d[J][K], eight FMAs.
template <typename T>
__device__ __forceinline__ void interp31(T d00, T d10, T d01, T d11, T (&o)[2][2]) {
    const T e00 = fma(T(3), d00, d10), e10 = fma(T(3), d10, d00);  // (b, K=0)
    const T e01 = fma(T(3), d01, d11), e11 = fma(T(3), d11, d01);  // (b, K=1)
    o[0][0] = fma(T(3), e00, e01);
    o[0][1] = fma(T(3), e01, e00);
    o[1][0] = fma(T(3), e10, e11);
    o[1][1] = fma(T(3), e11, e10);
}

// Displacement gradients of the cell's points from corner displacements held
// as u/32: the 3/1 weights then give (1/h) sum w w (difference) exactly.
template <typename T>
__device__ __forceinline__ void cell_gradients31(const T (&u)[8][3], CellGrad<T> &g) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        T o[2][2];
        interp31<T>(u[corner(1, 0, 0)][d] - u[corner(0, 0, 0)][d], u[corner(1, 1, 0)][d] - u[corner(0, 1, 0)][d],
                    u[corner(1, 0, 1)][d] - u[corner(0, 0, 1)][d], u[corner(1, 1, 1)][d] - u[corner(0, 1, 1)][d], o);
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) g.gx[b][c][d] = o[b][c];
        interp31<T>(u[corner(0, 1, 0)][d] - u[corner(0, 0, 0)][d], u[corner(1, 1, 0)][d] - u[corner(1, 0, 0)][d],
                    u[corner(0, 1, 1)][d] - u[corner(0, 0, 1)][d], u[corner(1, 1, 1)][d] - u[corner(1, 0, 1)][d], o);
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int c = 0; c < 2; ++c) g.gy[a][c][d] = o[a][c];
        interp31<T>(u[corner(0, 0, 1)][d] - u[corner(0, 0, 0)][d], u[corner(1, 0, 1)][d] - u[corner(1, 0, 0)][d],
                    u[corner(0, 1, 1)][d] - u[corner(0, 1, 0)][d], u[corner(1, 1, 1)][d] - u[corner(1, 1, 0)][d], o);
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) g.gz[a][b][d] = o[a][b];
    }
}

// Eight points of one cell: F[corner] = (2I-1) X'[J][K] + (2J-1) Y'[I][K] +
// (2K-1) Z'[I][J] with X', Y', Z' the 3/1-weighted sums of the traction
// columns of sigma; the nodal force is -(V/h)/16 F = -F/32 (V = 1 voxel, h = 2).
template <typename T>
__device__ __forceinline__ void cell_forces(const T (&u)[8][3], const uint4 &sp, const T *__restrict__ ctab,
                                            const T (&eb)[6], T (&f)[8][3]) {
    CellGrad<T> g;
    cell_gradients31<T>(u, g);
    T tx[2][2][3], ty[2][2][3], tz[2][2][3];  // traction sums over a, b, c respectively
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int d = 0; d < 3; ++d) tx[i][j][d] = ty[i][j][d] = tz[i][j][d] = T(0);
    Row24<T> row;
    uint32_t qprev = 0xffffffffu;
#pragma unroll
    for (int L = 0; L < 8; ++L) {
        const int a = L & 1, b = (L >> 1) & 1, c = L >> 2;
        T e[6], s[6];
        point_strain<T>(g, eb, a, b, c, e);
        // points of one cell mostly share one orientation: fetch the row only when it changes
        const uint32_t q = spin_of(sp, local_slot(L));
        if (q != qprev) {
            row.load(ctab + 24ll * q);
            qprev = q;
        }
        hooke21<T>(row.v, e, s);
        // columns of sigma: x = (s0,s5,s4), y = (s5,s1,s3), z = (s4,s3,s2)
        tx[b][c][0] += s[0]; tx[b][c][1] += s[5]; tx[b][c][2] += s[4];
        ty[a][c][0] += s[5]; ty[a][c][1] += s[1]; ty[a][c][2] += s[3];
        tz[a][b][0] += s[4]; tz[a][b][1] += s[3]; tz[a][b][2] += s[2];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        T X[2][2], Y[2][2], Z[2][2];
        interp31<T>(tx[0][0][d], tx[1][0][d], tx[0][1][d], tx[1][1][d], X);  // X[J][K]
        interp31<T>(ty[0][0][d], ty[1][0][d], ty[0][1][d], ty[1][1][d], Y);  // Y[I][K]
        interp31<T>(tz[0][0][d], tz[1][0][d], tz[0][1][d], tz[1][1][d], Z);  // Z[I][J]
#pragma unroll
        for (int K = 0; K < 2; ++K)
#pragma unroll
            for (int J = 0; J < 2; ++J)
#pragma unroll
                for (int I = 0; I < 2; ++I) {
                    const T fx = I ? X[J][K] : -X[J][K];
                    const T fy = J ? Y[I][K] : -Y[I][K];
                    const T fz = K ? Z[I][J] : -Z[I][J];
                    f[corner(I, J, K)][d] = fx + fy + fz;
                }
    }
}

template <typename T>
__global__ void __launch_bounds__(NTHR, (sizeof(T) == 4 ? 2 : 1)) k_mpm_step(MpmArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MpmSmem<T> &sm = *reinterpret_cast<MpmSmem<T> *>(smem_raw);
    const int tid = threadIdx.x;
    const int lci = tid % CT, lcj = tid / CT;           // this thread's cell in the patch
    const long long plane = (long long)a.nbx * a.nby;
    const T fscale = -a.dt_over_m * T(0.03125);          // -dt / (32 m)
    T eb[6];
    load_ebar<T>(a.st, eb);
    // this CTA's contiguous range of the linear (tile, plane) index
    const long long total = (long long)a.tiles_x * a.tiles_y * a.nbz;
    long long w = total * blockIdx.x / gridDim.x;
    const long long wend = total * (blockIdx.x + 1) / gridDim.x;
    while (w < wend) {
        const int tile = (int)(w / a.nbz);
        const int k0 = (int)(w % a.nbz);
        const int kend = (int)min((long long)a.nbz, (long long)k0 + (wend - w));
        w += kend - k0;
        const int i0 = (tile % a.tiles_x) * OT, j0 = (tile / a.tiles_x) * OT;
        const int ni = i0 - 1 + lci, nj = j0 - 1 + lcj;      // node at the cell's lower corner
        const bool own = lci >= 1 && lcj >= 1 && ni < a.nbx && nj < a.nby;
        // a cell is needed when some owned node uses it: local index <= last owned local index
        const bool need = lci <= min(OT, a.nbx - i0) && lcj <= min(OT, a.nby - j0);
        const int gi = wrapi(ni, a.nbx), gj = wrapi(nj, a.nby);
        const long long col = gi + (long long)a.nbx * gj;   // (i, j) column offset of cell and node

        int b0 = 0, b1 = 1, b2 = 2;
        load_plane<T>(sm, b0, a.u_in, i0, j0, k0 - 1, a.nbx, a.nby, a.nbz);
        load_plane<T>(sm, b1, a.u_in, i0, j0, k0, a.nbx, a.nby, a.nbz);
        uint4 sp = need ? __ldg(a.spins + col + plane * wrapi(k0 - 1, a.nbz)) : make_uint4(0, 0, 0, 0);
        __syncthreads();

        T acc[3] = {T(0), T(0), T(0)};
        for (int kk = k0 - 1; kk < kend; ++kk) {
            // one plane ahead: next plane's spins, this plane's owned velocity, plane kk+2 of u
            uint4 sp_next = make_uint4(0, 0, 0, 0);
            if (need && kk + 1 < kend) sp_next = __ldg(a.spins + col + plane * (kk + 1));
            T vold[3] = {T(0), T(0), T(0)};
            const long long nidx = 3ll * (col + plane * (long long)(kk < 0 ? 0 : kk));
            if (own && kk >= k0) {
#pragma unroll
                for (int d = 0; d < 3; ++d) vold[d] = a.v[nidx + d];
            }
            if (kk + 1 < kend) load_plane<T>(sm, b2, a.u_in, i0, j0, kk + 2, a.nbx, a.nby, a.nbz);
            if (need) {
                T u[8][3];
#pragma unroll
                for (int K = 0; K < 2; ++K)
#pragma unroll
                    for (int J = 0; J < 2; ++J)
#pragma unroll
                        for (int I = 0; I < 2; ++I)
#pragma unroll
                            for (int d = 0; d < 3; ++d) u[corner(I, J, K)][d] = sm.us[K ? b1 : b0][d][lcj + J][lci + I];
                T f[8][3];
                cell_forces<T>(u, sp, a.ctab, eb, f);
#pragma unroll
                for (int J = 0; J < 2; ++J)
#pragma unroll
                    for (int I = 0; I < 2; ++I)
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            sm.fb[I + 2 * J][d][lcj][lci] = f[corner(I, J, 0)][d];
                            sm.ft[I + 2 * J][d][lcj][lci] = f[corner(I, J, 1)][d];
                        }
            }
            __syncthreads();
            if (own) {
                // cells (lci-1, lcj-1), (lci, lcj-1), (lci-1, lcj), (lci, lcj) see this node as corner 3, 2, 1, 0
                if (kk >= k0) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const T F = acc[d] + sm.fb[3][d][lcj - 1][lci - 1] + sm.fb[2][d][lcj - 1][lci] +
                                    sm.fb[1][d][lcj][lci - 1] + sm.fb[0][d][lcj][lci];
                        const T vn = a.keep * vold[d] + fscale * F;
                        a.v[nidx + d] = vn;
                        a.u_out[nidx + d] = sm.us[b0][d][lcj][lci] * T(32) + a.dt * vn;
                    }
                }
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    acc[d] = sm.ft[3][d][lcj - 1][lci - 1] + sm.ft[2][d][lcj - 1][lci] + sm.ft[1][d][lcj][lci - 1] +
                             sm.ft[0][d][lcj][lci];
            }
            __syncthreads();
            const int t = b0;
            b0 = b1;
            b1 = b2;
            b2 = t;
            sp = sp_next;
        }
    }
}

}  // namespace

int mpm_tiles(int nb) { return (nb + OT - 1) / OT; }

cudaError_t mpm_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_mpm_step<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(MpmSmem<float>));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_mpm_step<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(MpmSmem<double>));
}

// Persistent grid: resident CTAs per SM x SMs, but at least four planes per CTA.
template <typename T>
int mpm_grid(int nbx, int nby, int nbz, int num_sms) {
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mpm_step<T>, NTHR, sizeof(MpmSmem<T>)) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const long long planes = (long long)mpm_tiles(nbx) * mpm_tiles(nby) * nbz;
    long long g = (long long)per_sm * num_sms;
    const long long cap = (planes + 3) / 4;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}
template int mpm_grid<float>(int, int, int, int);
template int mpm_grid<double>(int, int, int, int);

template <typename T>
cudaError_t launch_mpm_step(const MpmArgs<T> &a, cudaStream_t s) {
    k_mpm_step<T><<<a.grid, NTHR, sizeof(MpmSmem<T>), s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_mpm_step<float>(const MpmArgs<float> &, cudaStream_t);
template cudaError_t launch_mpm_step<double>(const MpmArgs<double> &, cudaStream_t);

}  // namespace hmc
