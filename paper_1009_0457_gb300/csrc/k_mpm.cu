// Fused explicit MPM step (Sec. "Elastic Deformation"): for every material
// point strain from the nodal displacement, Hooke's law (Eq. 1) with the
// point's rotated stiffness, internal nodal force, then the damped
// velocity / displacement update of every node -- one kernel, one pass over
// the spins and the nodal state.
//
// Tiling: a CTA of 16x16 threads owns a 16x16 column of nodes and marches up
// a chunk of node planes in z.  For every cell plane it computes the 17x17
// cells that touch its nodes (one cell ring of halo in x and y), each cell's
// eight points in one thread, and writes each cell's eight nodal force
// contributions to shared memory; a node's force is then the sum of its four
// cells below and four cells above, the latter carried in registers from the
// previous plane.  Displacements are read from one buffer and written to the
// other, so CTAs never race on the halo.
#include "hmc_device.cuh"

namespace hmc {

namespace {

constexpr int TX = 16, TY = 16, CX = TX + 1, CY = TY + 1, NXS = TX + 2, NYS = TY + 2;
constexpr int NTHR = TX * TY;

template <typename T>
struct MpmSmem {
    T us[2][NYS][NXS][3];  // node planes kk and kk+1 (with one node of halo on each side)
    T fb[CY][CX][4][3];    // cell contributions to their four lower nodes (plane kk)
    T ft[CY][CX][4][3];    // cell contributions to their four upper nodes (plane kk+1)
};

template <typename T>
__device__ __forceinline__ void load_plane(MpmSmem<T> &sm, int slot, const T *__restrict__ u, int i0, int j0,
                                           int k, int nbx, int nby, int nbz) {
    const int gk = wrapi(k, nbz);
    for (int t = threadIdx.x; t < NYS * NXS; t += NTHR) {
        const int li = t % NXS, lj = t / NXS;
        const int gi = wrapi(i0 - 1 + li, nbx), gj = wrapi(j0 - 1 + lj, nby);
        const long long n = 3ll * (gi + (long long)nbx * (gj + (long long)nby * gk));
        sm.us[slot][lj][li][0] = u[n];
        sm.us[slot][lj][li][1] = u[n + 1];
        sm.us[slot][lj][li][2] = u[n + 2];
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
#pragma unroll
    for (int L = 0; L < 8; ++L) {
        const int a = L & 1, b = (L >> 1) & 1, c = L >> 2;
        T e[6], s[6];
        point_strain<T>(g, eb, a, b, c, e);
        Row24<T> row;
        row.load(ctab + 24ll * spin_of(sp, local_slot(L)));
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
    const int tx = tid % TX, ty = tid / TX;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k0 = blockIdx.z * a.zc;
    const int kend = min(k0 + a.zc, a.nbz);
    const int ni = i0 + tx, nj = j0 + ty;
    const bool own = ni < a.nbx && nj < a.nby;
    // cells needed by the owned nodes: local cell index lc = cell - (i0 - 1) <= last owned - i0 + 1
    const int lci_max = min(TX, a.nbx - i0), lcj_max = min(TY, a.nby - j0);
    T eb[6];
    load_ebar<T>(a.st, eb);

    int cur = 0;
    load_plane<T>(sm, 0, a.u_in, i0, j0, k0 - 1, a.nbx, a.nby, a.nbz);
    load_plane<T>(sm, 1, a.u_in, i0, j0, k0, a.nbx, a.nby, a.nbz);
    __syncthreads();

    T acc[3] = {T(0), T(0), T(0)};
    for (int kk = k0 - 1; kk < kend; ++kk) {
        const int gk = wrapi(kk, a.nbz);
        for (int c = tid; c < CX * CY; c += NTHR) {
            const int lci = c % CX, lcj = c / CX;
            if (lci > lci_max || lcj > lcj_max) continue;
            T u[8][3];
#pragma unroll
            for (int K = 0; K < 2; ++K)
#pragma unroll
                for (int J = 0; J < 2; ++J)
#pragma unroll
                    for (int I = 0; I < 2; ++I)
#pragma unroll
                        for (int d = 0; d < 3; ++d) u[corner(I, J, K)][d] = sm.us[cur ^ K][lcj + J][lci + I][d];
            const int gi = wrapi(i0 - 1 + lci, a.nbx), gj = wrapi(j0 - 1 + lcj, a.nby);
            const uint4 sp = __ldg(a.spins + (gi + (long long)a.nbx * (gj + (long long)a.nby * gk)));
            T f[8][3];
            cell_forces<T>(u, sp, a.ctab, eb, f);
#pragma unroll
            for (int J = 0; J < 2; ++J)
#pragma unroll
                for (int I = 0; I < 2; ++I)
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        sm.fb[lcj][lci][I + 2 * J][d] = f[corner(I, J, 0)][d];
                        sm.ft[lcj][lci][I + 2 * J][d] = f[corner(I, J, 1)][d];
                    }
        }
        __syncthreads();
        if (own) {
            if (kk >= k0) {
                const long long n = 3ll * (ni + (long long)a.nbx * (nj + (long long)a.nby * kk));
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const T f = acc[d] + sm.fb[ty][tx][3][d] + sm.fb[ty][tx + 1][2][d] + sm.fb[ty + 1][tx][1][d] +
                                sm.fb[ty + 1][tx + 1][0][d];
                    const T vn = a.keep * a.v[n + d] + a.dt_over_m * f;
                    a.v[n + d] = vn;
                    a.u_out[n + d] = sm.us[cur][ty + 1][tx + 1][d] + a.dt * vn;
                }
            }
#pragma unroll
            for (int d = 0; d < 3; ++d)
                acc[d] = sm.ft[ty][tx][3][d] + sm.ft[ty][tx + 1][2][d] + sm.ft[ty + 1][tx][1][d] +
                         sm.ft[ty + 1][tx + 1][0][d];
        }
        __syncthreads();
        if (kk + 1 < kend) load_plane<T>(sm, cur, a.u_in, i0, j0, kk + 2, a.nbx, a.nby, a.nbz);
        cur ^= 1;
        __syncthreads();
    }
}

}  // namespace

int mpm_zchunk(int nbx, int nby, int nbz, int num_sms) {
    // enough CTAs for several waves of two resident CTAs per SM, but chunks of
    // at least 4 planes so the one-plane z halo stays a small overhead
    const long long tiles = (long long)((nbx + TX - 1) / TX) * ((nby + TY - 1) / TY);
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
    dim3 grid((a.nbx + TX - 1) / TX, (a.nby + TY - 1) / TY, (a.nbz + a.zc - 1) / a.zc);
    k_mpm_step<T><<<grid, NTHR, smem, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_mpm_step<float>(const MpmArgs<float> &, cudaStream_t);
template cudaError_t launch_mpm_step<double>(const MpmArgs<double> &, cudaStream_t);

}  // namespace hmc
