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
        sm.us[buf][0][lj][li] = __ldg(u + n);
        sm.us[buf][1][lj][li] = __ldg(u + n + 1);
        sm.us[buf][2][lj][li] = __ldg(u + n + 2);
    }
}

// Eight points of one cell: forces on its corner nodes, -(V/h) times the
// separable sums of the traction columns of sigma (V = 1 voxel, h = 2).
template <typename T>
__device__ __forceinline__ void cell_forces(const T (&u)[8][3], const uint4 &sp, const T *__restrict__ ctab,
                                            const T (&eb)[6], T (&f)[8][3]) {
    CellGrad<T> g;
    cell_gradients<T>(u, g);
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
        interp2<T>(tx[0][0][d], tx[1][0][d], tx[0][1][d], tx[1][1][d], X);  // X[J][K]
        interp2<T>(ty[0][0][d], ty[1][0][d], ty[0][1][d], ty[1][1][d], Y);  // Y[I][K]
        interp2<T>(tz[0][0][d], tz[1][0][d], tz[0][1][d], tz[1][1][d], Z);  // Z[I][J]
#pragma unroll
        for (int K = 0; K < 2; ++K)
#pragma unroll
            for (int J = 0; J < 2; ++J)
#pragma unroll
                for (int I = 0; I < 2; ++I) {
                    const T fx = I ? X[J][K] : -X[J][K];
                    const T fy = J ? Y[I][K] : -Y[I][K];
                    const T fz = K ? Z[I][J] : -Z[I][J];
                    f[corner(I, J, K)][d] = -(fx + fy + fz);
                }
    }
}

template <typename T>
__global__ void __launch_bounds__(NTHR, (sizeof(T) == 4 ? 2 : 1)) k_mpm_step(MpmArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MpmSmem<T> &sm = *reinterpret_cast<MpmSmem<T> *>(smem_raw);
    const int tid = threadIdx.x;
    const int lci = tid % CT, lcj = tid / CT;           // this thread's cell in the patch
    const int i0 = blockIdx.x * OT, j0 = blockIdx.y * OT, k0 = blockIdx.z * a.zc;
    const int kend = min(k0 + a.zc, a.nbz);
    const int ni = i0 - 1 + lci, nj = j0 - 1 + lcj;      // node at the cell's lower corner
    const bool own = lci >= 1 && lcj >= 1 && ni < a.nbx && nj < a.nby;
    // a cell is needed when some owned node uses it: local index <= last owned local index
    const bool need = lci <= min(OT, a.nbx - i0) && lcj <= min(OT, a.nby - j0);
    const int gi = wrapi(ni, a.nbx), gj = wrapi(nj, a.nby);
    const long long col = gi + (long long)a.nbx * gj;   // (i, j) column offset of cell and node
    const long long plane = (long long)a.nbx * a.nby;
    T eb[6];
    load_ebar<T>(a.st, eb);

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
                    const T f = acc[d] + sm.fb[3][d][lcj - 1][lci - 1] + sm.fb[2][d][lcj - 1][lci] +
                                sm.fb[1][d][lcj][lci - 1] + sm.fb[0][d][lcj][lci];
                    const T vn = a.keep * vold[d] + a.dt_over_m * f;
                    a.v[nidx + d] = vn;
                    a.u_out[nidx + d] = sm.us[b0][d][lcj][lci] + a.dt * vn;
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

}  // namespace

int mpm_zchunk(int nbx, int nby, int nbz, int num_sms) {
    // enough CTAs for several waves of two resident CTAs per SM, but chunks of
    // at least 4 planes so the one-plane z halo stays a small overhead
    const long long tiles = (long long)((nbx + OT - 1) / OT) * ((nby + OT - 1) / OT);
    const long long target = 8ll * num_sms;
    long long chunks = (target + tiles - 1) / tiles;
    int zc = (int)((nbz + chunks - 1) / chunks);
    if (zc < 4) zc = 4;
    if (zc > nbz) zc = nbz;
    return zc;
}

cudaError_t mpm_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_mpm_step<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(MpmSmem<float>));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_mpm_step<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(MpmSmem<double>));
}

template <typename T>
cudaError_t launch_mpm_step(const MpmArgs<T> &a, cudaStream_t s) {
    const size_t smem = sizeof(MpmSmem<T>);
    dim3 grid((a.nbx + OT - 1) / OT, (a.nby + OT - 1) / OT, (a.nbz + a.zc - 1) / a.zc);
    k_mpm_step<T><<<grid, NTHR, smem, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_mpm_step<float>(const MpmArgs<float> &, cudaStream_t);
template cudaError_t launch_mpm_step<double>(const MpmArgs<double> &, cudaStream_t);

}  // namespace hmc
