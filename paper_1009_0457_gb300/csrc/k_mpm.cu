// Fused explicit MPM step (Sec. "Elastic Deformation"): for every material
// point strain from the nodal displacement, Hooke's law (Eq. 1) with the
// point's rotated stiffness, internal nodal force, then the damped
// velocity / displacement update of every node -- one kernel, one pass over
// the spins and the nodal state.
//
// Tiling: a CTA of CX x CY threads (16x16, 32x8 or 8x32, chosen per batch by
// the autotuner) computes a CX x CY patch of cells per cell plane (one thread
// per cell, all eight points of the cell) and owns the (CX-1) x (CY-1) nodes
// whose four lower and four upper cells all lie in the patch.  It
// marches up a chunk of planes in z: each cell writes its eight nodal force
// contributions to shared memory, and a node's force is the sum of its four
// cells below (carried in registers from the previous plane) and four above.
// Node planes are triple-buffered in shared memory (structure of arrays, so
// neighbouring threads hit neighbouring banks) and the next plane's spins and
// the owned node's velocity are fetched one plane ahead.  Displacements are
// read from one buffer and written to the other, so CTAs never race on the halo.
//
// Scheduling: the (replica, tile, plane) space of the whole batch is cut into
// one contiguous range per resident CTA (a persistent grid of occupancy x
// SMs), so every CTA marches about the same number of planes, over replicas of
// any size, and pays the one-plane restart only where its range enters a new
// tile.  In a tile cut by a replica's high edges the needed cells are numbered
// so that the active threads fill whole warps.  The next node plane is read into registers before the cells of the
// current plane are computed and stored to shared memory after them.
//
// Scaling: the interpolation weights 3/4 and 1/4 of the trilinear shape
// functions at the points 1/4 and 3/4 of the cell are applied as 3 and 1; the
// factors 1/16 and 1/h are folded into the displacements held in shared memory
// (u/32) and into the force constant of the node update (-dt/(32 m)) -- both
// exact powers of two.
#include "hmc_device.cuh"

namespace hmc {

namespace {

// A node's or a cell corner's three components and a pad: one 16-byte shared-memory access
// in FP32 (eight consecutive lanes read 128 contiguous bytes, free of bank conflicts)
// instead of three 4-byte ones.
template <typename T>
struct alignas(16) Vec4 {
    T x, y, z, p;
};

template <int CX, int CY>
struct MpmSmem {
    static constexpr int NX = CX + 1, NY = CY + 1;   // node tile (one node of halo each side)
    template <typename T>
    struct S {
        Vec4<T> us[3][NY][NX];  // node planes (buffer, j, i), held as u/32
        Vec4<T> fb[4][CY][CX];  // cell contributions to their lower corner nodes (corner I+2J)
        Vec4<T> ft[4][CY][CX];  // ... to their upper corner nodes
    };
};

// byte offset of the FP32 orientation table behind a CTA's tiles (16-byte aligned)
template <int CX, int CY, typename T>
__host__ __device__ constexpr size_t mpm_table_offset() {
    return (sizeof(typename MpmSmem<CX, CY>::template S<T>) + 15) & ~size_t(15);
}

// Node plane k of the tile with origin (i0, j0) (one node of halo on each side),
// read from global memory into registers / written to shared memory.
template <typename T, int CX, int CY>
struct PlaneLoad {
    static constexpr int NX = CX + 1, NY = CY + 1, NN = NX * NY, NTHR = CX * CY;
    static constexpr int PER = (NN + NTHR - 1) / NTHR;
    T r[PER][3];
    int col[PER];   // this thread's tile nodes as (i + nbx j) in the replica's node plane
    // once per tile: the periodic (i, j) of each node this thread loads
    __device__ __forceinline__ void prepare(int i0, int j0, int nbx, int nby) {
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int t = threadIdx.x + m * NTHR;
            const int li = t % NX, lj = t / NX;
            col[m] = wrapi(i0 - 1 + li, nbx) + nbx * wrapi(j0 - 1 + lj, nby);
        }
    }
    // node plane k, -1 <= k <= nbz (periodic in z)
    __device__ __forceinline__ void fetch(const T *__restrict__ u, long long node0, int k, int nbz, int plane) {
        const int gk = k < 0 ? k + nbz : (k >= nbz ? k - nbz : k);
        const T *base = u + 3 * (node0 + (long long)plane * gk);
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int t = threadIdx.x + m * NTHR;
            if (t < NN) {
                const T *p = base + 3 * col[m];
                r[m][0] = __ldg(p);
                r[m][1] = __ldg(p + 1);
                r[m][2] = __ldg(p + 2);
            }
        }
    }
    __device__ __forceinline__ void store(Vec4<T> (&us)[NY][NX]) const {
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int t = threadIdx.x + m * NTHR;
            if (t < NN)   // node (t % NX, t / NX) of the row-major tile
                (&us[0][0])[t] = Vec4<T>{r[m][0] * T(0.03125), r[m][1] * T(0.03125), r[m][2] * T(0.03125), T(0)};
        }
    }
};

// Hooke's law for the MPM step.  FP64: the 21-entry symmetric row of C'(q).  FP32:
// the cubic form of one rotated cubic material,
//   sigma = (C12 tr + Ad p2) I + 2 C44 eps + Ad (p0 - p2) a0 a0 + Ad (p1 - p2) a1 a1,
//   p_m = a_m.eps.a_m = W_m.e,  p2 = tr - p0 - p1,  Ad = C11 - C12 - 2 C44,
// with e the Voigt strain (engineering shear), sigma in tensor shear and W_m the Voigt
// weights (x^2, y^2, z^2, yz, xz, xy) of crystal axis a_m = (x, y, z); the third axis
// drops out because the axes are orthonormal.  12 values per orientation instead of
// 21, so the table of up to MPM_STAB_MAX orientations sits in shared memory (STAB) and
// a cell whose points change orientation reloads from there.  Every operation is
// explicitly rounded, in one order, in the scalar form and in the paired forms
// (__ffma2_rn: two FP32 FMAs per instruction), which therefore give the same bits.
__device__ __forceinline__ void cubic_hooke(const float (&w)[12], const float (&cub)[4], const float (&e)[6],
                                            float (&s)[6]) {
    float p0 = __fmul_rn(w[0], e[0]), p1 = __fmul_rn(w[6], e[0]);
#pragma unroll
    for (int k = 1; k < 6; ++k) {
        p0 = __fmaf_rn(w[k], e[k], p0);
        p1 = __fmaf_rn(w[6 + k], e[k], p1);
    }
    const float tr = __fadd_rn(__fadd_rn(e[0], e[1]), e[2]);
    const float p2 = __fsub_rn(__fsub_rn(tr, p0), p1);
    // A = Ad p2; c = C12 tr + A; d_m = Ad p_m - A (one fused operation each)
    const float A = __fmul_rn(cub[3], p2);
    const float c = __fmaf_rn(cub[0], tr, A);
    const float d0 = __fmaf_rn(cub[3], p0, -A), d1 = __fmaf_rn(cub[3], p1, -A);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float base = k < 3 ? __fmaf_rn(cub[1], e[k], c) : __fmul_rn(cub[2], e[k]);
        s[k] = __fmaf_rn(d1, w[6 + k], __fmaf_rn(d0, w[k], base));
    }
}

// the same with the two axis products and the stress components formed in pairs
__device__ __forceinline__ void cubic_hooke_paired(const float (&w)[12], const float (&cub)[4], const float (&e)[6],
                                                   float (&s)[6]) {
    float2 pp = __fmul2_rn(make_float2(w[0], w[6]), make_float2(e[0], e[0]));
#pragma unroll
    for (int k = 1; k < 6; ++k) pp = __ffma2_rn(make_float2(w[k], w[6 + k]), make_float2(e[k], e[k]), pp);
    const float p0 = pp.x, p1 = pp.y;
    const float tr = __fadd_rn(__fadd_rn(e[0], e[1]), e[2]);
    const float p2 = __fsub_rn(__fsub_rn(tr, p0), p1);
    const float A = __fmul_rn(cub[3], p2);
    const float c = __fmaf_rn(cub[0], tr, A);
    const float2 dd = __ffma2_rn(make_float2(cub[3], cub[3]), pp, make_float2(-A, -A));
    const float d0 = dd.x, d1 = dd.y;
    const float2 D0 = make_float2(d0, d0), D1 = make_float2(d1, d1);
    float2 base[3];
    base[0] = __ffma2_rn(make_float2(cub[1], cub[1]), make_float2(e[0], e[1]), make_float2(c, c));
    base[1] = make_float2(__fmaf_rn(cub[1], e[2], c), __fmul_rn(cub[2], e[3]));
    base[2] = __fmul2_rn(make_float2(cub[2], cub[2]), make_float2(e[4], e[5]));
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float2 t = __ffma2_rn(D0, make_float2(w[2 * j], w[2 * j + 1]), base[j]);
        const float2 r = __ffma2_rn(D1, make_float2(w[6 + 2 * j], w[7 + 2 * j]), t);
        s[2 * j] = r.x;
        s[2 * j + 1] = r.y;
    }
}

template <typename T, bool PAIR, bool STAB>
struct HookeRow {
    Row24<T> r;
    __device__ __forceinline__ void load(const T *tab, const float *, uint32_t q) { r.load(tab + 24ll * q); }
    __device__ __forceinline__ void apply(const T (&e)[6], T (&s)[6], const float (&)[4]) const {
        hooke21<T>(r.v, e, s);
    }
};
template <bool PAIR, bool STAB>
struct HookeRow<float, PAIR, STAB> {
    float w[12];
    // cw: the table in shared memory (STAB) or in global memory
    __device__ __forceinline__ void load(const float *, const float *cw, uint32_t q) {
        const float4 *p = reinterpret_cast<const float4 *>(cw + 12 * q);
        float4 v[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) v[i] = STAB ? p[i] : __ldg(p + i);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            w[4 * i] = v[i].x; w[4 * i + 1] = v[i].y; w[4 * i + 2] = v[i].z; w[4 * i + 3] = v[i].w;
        }
    }
    __device__ __forceinline__ void apply(const float (&e)[6], float (&s)[6], const float (&cub)[4]) const {
        if (PAIR)
            cubic_hooke_paired(w, cub, e, s);
        else
            cubic_hooke(w, cub, e, s);
    }
};

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

// The point visited n-th in a cell: the corners in a Gray-code order, one coordinate
// changing per step.  A cell split by a grain boundary reloads its stiffness row
// whenever the orientation changes from one point to the next: 4, 2 and 1 times for a
// boundary plane normal to x, y and z (7, 3 and 1 in plain corner order).  Every MPM
// variant visits the points in this order, so their results stay bit-identical.
__host__ __device__ constexpr int gray_point(int n) {
    return n == 0 ? 0 : n == 1 ? 1 : n == 2 ? 3 : n == 3 ? 2 : n == 4 ? 6 : n == 5 ? 7 : n == 6 ? 5 : 4;
}

// Eight points of one cell: F[corner] = (2I-1) X'[J][K] + (2J-1) Y'[I][K] +
// (2K-1) Z'[I][J] with X', Y', Z' the 3/1-weighted sums of the traction
// columns of sigma; the nodal force is -(V/h)/16 F = -F/32 (V = 1 voxel, h = 2).
template <typename T, bool PAIR, bool STAB>
__device__ __forceinline__ void cell_forces(const T (&u)[8][3], const uint4 &sp, const T *__restrict__ ctab,
                                            const float *cw, const float (&cub)[4], const T (&eb)[6],
                                            T (&f)[8][3]) {
    // the first point's stiffness row is requested before the gradients are formed, so that
    // its load latency overlaps them
    HookeRow<T, PAIR, STAB> row;
    uint32_t qprev = spin_of(sp, local_slot(0));
    row.load(ctab, cw, qprev);
    CellGrad<T> g;
    cell_gradients31<T>(u, g);
    // each strain component of a point is eb_k plus gradient entries that two points share:
    // add eb_k once to the one entry of each component that only that component uses (the
    // normal entries, and one of the two entries of each shear)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            g.gx[i][j][0] = eb[0] + g.gx[i][j][0];
            g.gy[i][j][1] = eb[1] + g.gy[i][j][1];
            g.gz[i][j][2] = eb[2] + g.gz[i][j][2];
            g.gz[i][j][1] = eb[3] + g.gz[i][j][1];
            g.gz[i][j][0] = eb[4] + g.gz[i][j][0];
            g.gy[i][j][0] = eb[5] + g.gy[i][j][0];
        }
    T tx[2][2][3], ty[2][2][3], tz[2][2][3];  // traction sums over a, b, c respectively
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int d = 0; d < 3; ++d) tx[i][j][d] = ty[i][j][d] = tz[i][j][d] = T(0);
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        const int L = gray_point(n);
        const int a = L & 1, b = (L >> 1) & 1, c = L >> 2;
        T e[6], s[6];
        e[0] = g.gx[b][c][0];
        e[1] = g.gy[a][c][1];
        e[2] = g.gz[a][b][2];
        e[3] = g.gz[a][b][1] + g.gy[a][c][2];
        e[4] = g.gz[a][b][0] + g.gx[b][c][2];
        e[5] = g.gy[a][c][0] + g.gx[b][c][1];
        // points of one cell mostly share one orientation: fetch the row only when it changes
        const uint32_t q = spin_of(sp, local_slot(L));
        if (q != qprev) {
            row.load(ctab, cw, q);
            qprev = q;
        }
        row.apply(e, s, cub);
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

template <typename T, int CX, int CY, bool PAIR, bool STAB>
__global__ void __launch_bounds__(CX *CY, (sizeof(T) == 4 ? 2 : 1)) k_mpm_step(MpmArgs<T> a) {
    constexpr int OX = CX - 1, OY = CY - 1;
    using Smem = typename MpmSmem<CX, CY>::template S<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    const int tid = threadIdx.x;
    const T fscale = -a.dt_over_m * T(0.03125);          // -dt / (32 m)
    // the next step may be launched now: its CTAs take the SM slots this grid's CTAs free
    // and stage their table while this grid finishes
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // FP32: the orientation table of the cubic form, staged in shared memory behind the tiles
    const float *cw = a.cubw;
    if constexpr (STAB) {
        float *ts = reinterpret_cast<float *>(smem_raw + mpm_table_offset<CX, CY, T>());
        for (int i = tid; i < 3 * a.nq; i += CX * CY)
            reinterpret_cast<float4 *>(ts)[i] = __ldg(reinterpret_cast<const float4 *>(a.cubw) + i);
        __syncthreads();
        cw = ts;
    }
    float cub[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) cub[i] = a.cub[i];
    // everything above reads only constant tables; u, v, the spins and the mean strain come
    // from the kernels before this one
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // this CTA's contiguous range of the linear (replica, tile, plane) index
    long long w = a.total * blockIdx.x / gridDim.x;
    const long long wend = a.total * (blockIdx.x + 1) / gridDim.x;
    int r = 0;
    while (w < wend) {
        while (a.sched[r + 1].plane_off <= w) ++r;        // replica of work item w (ranges are ascending)
        const Replica &R = a.reps[r];
        const MpmSched &SC = a.sched[r];
        const int nbx = R.nbx, nby = R.nby, nbz = R.nbz;
        const long long lw = w - SC.plane_off;
        const int tile = (int)(lw / nbz);
        const int k0 = (int)(lw - (long long)tile * nbz);
        const long long rem = min(wend, a.sched[r + 1].plane_off) - w;
        const int kend = (int)min((long long)nbz, (long long)k0 + rem);
        w += kend - k0;
        const int i0 = (tile % SC.tiles_x) * OX, j0 = (tile / SC.tiles_x) * OY;
        // cells needed by the tile's owned nodes: W x H (fewer at the high edges of the replica);
        // they are numbered W-wide so that the active threads fill whole warps
        const int W = min(CX, nbx - i0 + 1), H = min(CY, nby - j0 + 1);
        const int lci = tid % W, lcj = tid / W;               // this thread's cell in the patch
        const bool need = tid < W * H;
        const int ni = i0 - 1 + lci, nj = j0 - 1 + lcj;      // node at the cell's lower corner
        const bool own = need && lci >= 1 && lcj >= 1;
        const int gi = wrapi(ni, nbx), gj = wrapi(nj, nby);
        const int plane = nbx * nby;
        const long long col = R.blk_off + gi + nbx * gj;    // (i, j) column of this cell and node in the batch
        T eb[6];
        load_ebar<T>(R.st, eb);

        PlaneLoad<T, CX, CY> pl;
        int b0 = 0, b1 = 1, b2 = 2;
        pl.prepare(i0, j0, nbx, nby);
        pl.fetch(a.u_in, R.blk_off, k0 - 1, nbz, plane);
        pl.store(sm.us[b0]);
        pl.fetch(a.u_in, R.blk_off, k0, nbz, plane);
        pl.store(sm.us[b1]);
        uint4 sp = need ? __ldg(a.spins + col + (long long)plane * wrapi(k0 - 1, nbz)) : make_uint4(0, 0, 0, 0);
        __syncthreads();

        T acc[3] = {T(0), T(0), T(0)};
        // this column's spins of the next plane, and its node's velocity and new displacement in
        // the current plane, advanced by one plane per iteration
        const uint4 *spn = a.spins + col + (long long)plane * k0;
        T *vp = a.v + 3 * (col + (long long)plane * k0);
        T *up = a.u_out + 3 * (col + (long long)plane * k0);
        const long long pstride = 3ll * plane;
        for (int kk = k0 - 1; kk < kend; ++kk) {
            // one plane ahead: next plane's spins and u, this plane's owned velocity
            uint4 sp_next = make_uint4(0, 0, 0, 0);
            if (need && kk + 1 < kend) sp_next = __ldg(spn);
            spn += plane;
            T vold[3] = {T(0), T(0), T(0)};
            if (own && kk >= k0) {
#pragma unroll
                for (int d = 0; d < 3; ++d) vold[d] = vp[d];
            }
            const bool more = kk + 1 < kend;
            if (more) pl.fetch(a.u_in, R.blk_off, kk + 2, nbz, plane);
            if (need) {
                T u[8][3];
#pragma unroll
                for (int K = 0; K < 2; ++K)
#pragma unroll
                    for (int J = 0; J < 2; ++J)
#pragma unroll
                        for (int I = 0; I < 2; ++I) {
                            const Vec4<T> n = sm.us[K ? b1 : b0][lcj + J][lci + I];
                            u[corner(I, J, K)][0] = n.x;
                            u[corner(I, J, K)][1] = n.y;
                            u[corner(I, J, K)][2] = n.z;
                        }
                T f[8][3];
                cell_forces<T, PAIR, STAB>(u, sp, a.ctab, cw, cub, eb, f);
#pragma unroll
                for (int J = 0; J < 2; ++J)
#pragma unroll
                    for (int I = 0; I < 2; ++I) {
                        const T *fl = f[corner(I, J, 0)], *fu = f[corner(I, J, 1)];
                        sm.fb[I + 2 * J][lcj][lci] = Vec4<T>{fl[0], fl[1], fl[2], T(0)};
                        sm.ft[I + 2 * J][lcj][lci] = Vec4<T>{fu[0], fu[1], fu[2], T(0)};
                    }
            }
            if (more) pl.store(sm.us[b2]);   // buffer b2 was last read before the previous barrier
            __syncthreads();
            if (own) {
                // cells (lci-1, lcj-1), (lci, lcj-1), (lci-1, lcj), (lci, lcj) see this node as corner 3, 2, 1, 0
                if (kk >= k0) {
                    const Vec4<T> c3 = sm.fb[3][lcj - 1][lci - 1], c2 = sm.fb[2][lcj - 1][lci];
                    const Vec4<T> c1 = sm.fb[1][lcj][lci - 1], c0 = sm.fb[0][lcj][lci];
                    const Vec4<T> un = sm.us[b0][lcj][lci];
                    const T F[3] = {acc[0] + c3.x + c2.x + c1.x + c0.x, acc[1] + c3.y + c2.y + c1.y + c0.y,
                                    acc[2] + c3.z + c2.z + c1.z + c0.z};
                    const T uc[3] = {un.x, un.y, un.z};
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const T vn = rfma(fscale, F[d], rmul(a.keep, vold[d]));
                        vp[d] = vn;
                        up[d] = rfma(a.dt, vn, uc[d] * T(32));
                    }
                    vp += pstride;
                    up += pstride;
                }
                const Vec4<T> c3 = sm.ft[3][lcj - 1][lci - 1], c2 = sm.ft[2][lcj - 1][lci];
                const Vec4<T> c1 = sm.ft[1][lcj][lci - 1], c0 = sm.ft[0][lcj][lci];
                acc[0] = c3.x + c2.x + c1.x + c0.x;
                acc[1] = c3.y + c2.y + c1.y + c0.y;
                acc[2] = c3.z + c2.z + c1.z + c0.z;
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

// ---------------------------------------------------------------------------
// Two cells per thread.  Cells x and x+8 of a 16 x 16 patch are the two lanes of
// float2 registers, and every floating-point step of the cell is one paired
// instruction (__ffma2_rn, __fadd2_rn, __fmul2_rn) in the order and with the
// roundings of the one-cell kernel above, so the two kernels give the same
// bits.  128 threads per 16 x 16 patch, same tiles and schedule as the 16x16
// shape; node planes are held as pairs (u(k), u(k+8)) for k = 0..8.
// ---------------------------------------------------------------------------
struct MpmSmem2 {
    static constexpr int NY = 17, S2 = 24;   // node rows; pair columns (9 used), padded so that a
                                             // half-warp's two rows fall in disjoint banks
    float2 us[3][3][NY][S2];
    float2 fb[4][3][16][8];   // cell contributions (cell k, cell k+8) to their lower corner nodes
    float2 ft[4][3][16][8];   // ... to their upper corner nodes
};

__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __fadd2_rn(a, p_neg(b)); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }

__device__ __forceinline__ void interp31_2(float2 d00, float2 d10, float2 d01, float2 d11, float2 (&o)[2][2]) {
    const float2 three = make_float2(3.f, 3.f);
    const float2 e00 = p_fma(three, d00, d10), e10 = p_fma(three, d10, d00);
    const float2 e01 = p_fma(three, d01, d11), e11 = p_fma(three, d11, d01);
    o[0][0] = p_fma(three, e00, e01);
    o[0][1] = p_fma(three, e01, e00);
    o[1][0] = p_fma(three, e10, e11);
    o[1][1] = p_fma(three, e11, e10);
}

// The cubic form of Hooke's law (cubic_hooke) on two cells at once, every
// operation one paired instruction with the scalar form's rounding.
__device__ __forceinline__ void cubic_hooke2(const float2 (&w)[12], const float (&cub)[4], const float2 (&e)[6],
                                             float2 (&s)[6]) {
    float2 p0 = p_mul(w[0], e[0]), p1 = p_mul(w[6], e[0]);
#pragma unroll
    for (int k = 1; k < 6; ++k) {
        p0 = p_fma(w[k], e[k], p0);
        p1 = p_fma(w[6 + k], e[k], p1);
    }
    const float2 C12 = make_float2(cub[0], cub[0]), C44x2 = make_float2(cub[1], cub[1]);
    const float2 C44 = make_float2(cub[2], cub[2]), Ad = make_float2(cub[3], cub[3]);
    const float2 tr = p_add(p_add(e[0], e[1]), e[2]);
    const float2 p2 = p_sub(p_sub(tr, p0), p1);
    const float2 A = p_mul(Ad, p2);
    const float2 c = p_fma(C12, tr, A);
    const float2 d0 = p_fma(Ad, p0, p_neg(A)), d1 = p_fma(Ad, p1, p_neg(A));
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float2 base = k < 3 ? p_fma(C44x2, e[k], c) : p_mul(C44, e[k]);
        s[k] = p_fma(d1, w[6 + k], p_fma(d0, w[k], base));
    }
}

__device__ __forceinline__ void load_w_pair(const float *cw, uint32_t qa, uint32_t qb, float2 (&w)[12]) {
    const float4 *pa = reinterpret_cast<const float4 *>(cw + 12 * qa), *pb = reinterpret_cast<const float4 *>(cw + 12 * qb);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float4 x = __ldg(pa + i), y = __ldg(pb + i);
        w[4 * i] = make_float2(x.x, y.x);
        w[4 * i + 1] = make_float2(x.y, y.y);
        w[4 * i + 2] = make_float2(x.z, y.z);
        w[4 * i + 3] = make_float2(x.w, y.w);
    }
}

__device__ __forceinline__ void cell_forces2(const float2 (&u)[8][3], const uint4 &spa, const uint4 &spb,
                                             const float *__restrict__ cw, const float (&cub)[4],
                                             const float2 (&eb)[6], float2 (&f)[8][3]) {
    float2 row[12];
    uint32_t qa = spin_of(spa, local_slot(0)), qb = spin_of(spb, local_slot(0));
    load_w_pair(cw, qa, qb, row);
    float2 gx[2][2][3], gy[2][2][3], gz[2][2][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float2 o[2][2];
        interp31_2(p_sub(u[corner(1, 0, 0)][d], u[corner(0, 0, 0)][d]), p_sub(u[corner(1, 1, 0)][d], u[corner(0, 1, 0)][d]),
                   p_sub(u[corner(1, 0, 1)][d], u[corner(0, 0, 1)][d]), p_sub(u[corner(1, 1, 1)][d], u[corner(0, 1, 1)][d]), o);
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) gx[b][c][d] = o[b][c];
        interp31_2(p_sub(u[corner(0, 1, 0)][d], u[corner(0, 0, 0)][d]), p_sub(u[corner(1, 1, 0)][d], u[corner(1, 0, 0)][d]),
                   p_sub(u[corner(0, 1, 1)][d], u[corner(0, 0, 1)][d]), p_sub(u[corner(1, 1, 1)][d], u[corner(1, 0, 1)][d]), o);
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int c = 0; c < 2; ++c) gy[a][c][d] = o[a][c];
        interp31_2(p_sub(u[corner(0, 0, 1)][d], u[corner(0, 0, 0)][d]), p_sub(u[corner(1, 0, 1)][d], u[corner(1, 0, 0)][d]),
                   p_sub(u[corner(0, 1, 1)][d], u[corner(0, 1, 0)][d]), p_sub(u[corner(1, 1, 1)][d], u[corner(1, 1, 0)][d]), o);
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) gz[a][b][d] = o[a][b];
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            gx[i][j][0] = p_add(eb[0], gx[i][j][0]);
            gy[i][j][1] = p_add(eb[1], gy[i][j][1]);
            gz[i][j][2] = p_add(eb[2], gz[i][j][2]);
            gz[i][j][1] = p_add(eb[3], gz[i][j][1]);
            gz[i][j][0] = p_add(eb[4], gz[i][j][0]);
            gy[i][j][0] = p_add(eb[5], gy[i][j][0]);
        }
    float2 tx[2][2][3], ty[2][2][3], tz[2][2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int d = 0; d < 3; ++d) tx[i][j][d] = ty[i][j][d] = tz[i][j][d] = make_float2(0.f, 0.f);
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        const int L = gray_point(n);
        const int a = L & 1, b = (L >> 1) & 1, c = L >> 2;
        float2 e[6], s[6];
        e[0] = gx[b][c][0];
        e[1] = gy[a][c][1];
        e[2] = gz[a][b][2];
        e[3] = p_add(gz[a][b][1], gy[a][c][2]);
        e[4] = p_add(gz[a][b][0], gx[b][c][2]);
        e[5] = p_add(gy[a][c][0], gx[b][c][1]);
        const uint32_t na = spin_of(spa, local_slot(L)), nb = spin_of(spb, local_slot(L));
        if (na != qa || nb != qb) {
            load_w_pair(cw, na, nb, row);
            qa = na;
            qb = nb;
        }
        cubic_hooke2(row, cub, e, s);
        tx[b][c][0] = p_add(tx[b][c][0], s[0]); tx[b][c][1] = p_add(tx[b][c][1], s[5]); tx[b][c][2] = p_add(tx[b][c][2], s[4]);
        ty[a][c][0] = p_add(ty[a][c][0], s[5]); ty[a][c][1] = p_add(ty[a][c][1], s[1]); ty[a][c][2] = p_add(ty[a][c][2], s[3]);
        tz[a][b][0] = p_add(tz[a][b][0], s[4]); tz[a][b][1] = p_add(tz[a][b][1], s[3]); tz[a][b][2] = p_add(tz[a][b][2], s[2]);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float2 X[2][2], Y[2][2], Z[2][2];
        interp31_2(tx[0][0][d], tx[1][0][d], tx[0][1][d], tx[1][1][d], X);
        interp31_2(ty[0][0][d], ty[1][0][d], ty[0][1][d], ty[1][1][d], Y);
        interp31_2(tz[0][0][d], tz[1][0][d], tz[0][1][d], tz[1][1][d], Z);
#pragma unroll
        for (int K = 0; K < 2; ++K)
#pragma unroll
            for (int J = 0; J < 2; ++J)
#pragma unroll
                for (int I = 0; I < 2; ++I) {
                    const float2 fx = I ? X[J][K] : p_neg(X[J][K]);
                    const float2 fy = J ? Y[I][K] : p_neg(Y[I][K]);
                    const float2 fz = K ? Z[I][J] : p_neg(Z[I][J]);
                    f[corner(I, J, K)][d] = p_add(p_add(fx, fy), fz);
                }
    }
}

// float index of cell or node k (0..16) in a row of pairs (k, k+8)
__device__ __forceinline__ int pair_slot(int k) { return k < 8 ? 2 * k : 2 * (k - 8) + 1; }

// 4-byte global -> shared copies that complete asynchronously (no register staging)
__device__ __forceinline__ void cp_async4(float *smem_dst, const float *gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__global__ void __launch_bounds__(128, 2) k_mpm_step2(MpmArgs<float> a) {
    constexpr int CX = 16, CY = 16, OX = CX - 1, OY = CY - 1, NX = 17, NN = NX * NX, NT = 128;
    constexpr int PER = (NN + NT - 1) / NT;
    using S2 = MpmSmem2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S2 &sm = *reinterpret_cast<S2 *>(smem_raw);
    const int tid = threadIdx.x;
    const int tx = tid & 7, ty = tid >> 3;   // cells (tx, ty) and (tx + 8, ty) of the patch
    // The node planes hold u itself (the one-cell kernel holds u/32): strains, stresses and
    // forces here are 32 times those of the one-cell kernel, the mean strain is taken times 32
    // and the force constant over 32 -- exact powers of two, so every rounding is the same.
    const float fscale = -a.dt_over_m * 0.03125f * 0.03125f;
    long long w = a.total * blockIdx.x / gridDim.x;
    const long long wend = a.total * (blockIdx.x + 1) / gridDim.x;
    int r = 0;
    while (w < wend) {
        while (a.sched[r + 1].plane_off <= w) ++r;
        const Replica &R = a.reps[r];
        const MpmSched &SC = a.sched[r];
        const int nbx = R.nbx, nby = R.nby, nbz = R.nbz;
        const long long lw = w - SC.plane_off;
        const int tile = (int)(lw / nbz);
        const int k0 = (int)(lw - (long long)tile * nbz);
        const long long rem = min(wend, a.sched[r + 1].plane_off) - w;
        const int kend = (int)min((long long)nbz, (long long)k0 + rem);
        w += kend - k0;
        const int i0 = (tile % SC.tiles_x) * OX, j0 = (tile / SC.tiles_x) * OY;
        const int W = min(CX, nbx - i0 + 1), H = min(CY, nby - j0 + 1);
        const bool needa = tx < W && ty < H, needb = tx + 8 < W && ty < H;
        const int plane = nbx * nby;
        const long long cola = R.blk_off + wrapi(i0 - 1 + tx, nbx) + nbx * wrapi(j0 - 1 + ty, nby);
        const long long colb = R.blk_off + wrapi(i0 + 7 + tx, nbx) + nbx * wrapi(j0 - 1 + ty, nby);
        // owned nodes: (W-1) x (H-1), two per thread at most
        const int ow = W - 1, no = (W - 1) * (H - 1);
        int oi[2], oj[2];
        long long ocol[2];
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int n = tid + m * NT;
            oi[m] = 1 + n % ow;
            oj[m] = 1 + n / ow;
            ocol[m] = R.blk_off + wrapi(i0 - 1 + oi[m], nbx) + nbx * wrapi(j0 - 1 + oj[m], nby);
        }
        float2 eb[6];
        {
            float e1[6];
            load_ebar<float>(R.st, e1);
#pragma unroll
            for (int k = 0; k < 6; ++k) eb[k] = make_float2(32.f * e1[k], 32.f * e1[k]);
        }
        // node tile loads: node (li, lj) -> pair column li (lane x) and/or li - 8 (lane y)
        int pcol[PER];
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int t = tid + m * NT;
            pcol[m] = wrapi(i0 - 1 + t % NX, nbx) + nbx * wrapi(j0 - 1 + t / NX, nby);
        }
        // node plane k (-1 <= k <= nbz, periodic) into buffer b: node (li, lj) goes to pair li
        // (lane x) and/or pair li - 8 (lane y)
        auto fetch = [&](int k, int b) {
            const int gk = k < 0 ? k + nbz : (k >= nbz ? k - nbz : k);
            const float *base = a.u_in + 3 * (R.blk_off + (long long)plane * gk);
#pragma unroll
            for (int m = 0; m < PER; ++m) {
                const int t = tid + m * NT;
                if (t < NN) {
                    const int li = t % NX, lj = t / NX;
                    const float *src = base + 3 * pcol[m];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        float *row = reinterpret_cast<float *>(&sm.us[b][d][lj][0]);
                        if (li <= 8) cp_async4(row + 2 * li, src + d);
                        if (li >= 8) cp_async4(row + 2 * (li - 8) + 1, src + d);
                    }
                }
            }
            cp_async_commit();
        };
        int b0 = 0, b1 = 1, b2 = 2;
        fetch(k0 - 1, b0);
        fetch(k0, b1);
        cp_async_wait_all();
        uint4 spa = needa ? __ldg(a.spins + cola + (long long)plane * wrapi(k0 - 1, nbz)) : make_uint4(0, 0, 0, 0);
        uint4 spb = needb ? __ldg(a.spins + colb + (long long)plane * wrapi(k0 - 1, nbz)) : make_uint4(0, 0, 0, 0);
        __syncthreads();

        float acc[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        for (int kk = k0 - 1; kk < kend; ++kk) {
            uint4 spa_n = make_uint4(0, 0, 0, 0), spb_n = make_uint4(0, 0, 0, 0);
            if (kk + 1 < kend) {
                if (needa) spa_n = __ldg(a.spins + cola + (long long)plane * (kk + 1));
                if (needb) spb_n = __ldg(a.spins + colb + (long long)plane * (kk + 1));
            }
            float vold[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
            const long long poff = (long long)plane * (kk < 0 ? 0 : kk);
            if (kk >= k0) {
#pragma unroll
                for (int m = 0; m < 2; ++m)
                    if (tid + m * NT < no)
#pragma unroll
                        for (int d = 0; d < 3; ++d) vold[m][d] = a.v[3 * (ocol[m] + poff) + d];
            }
            const bool more = kk + 1 < kend;
            if (more) fetch(kk + 2, b2);   // b2 was last read before the previous plane's second barrier
            if (needa || needb) {
                float2 u[8][3];
#pragma unroll
                for (int K = 0; K < 2; ++K)
#pragma unroll
                    for (int J = 0; J < 2; ++J)
#pragma unroll
                        for (int I = 0; I < 2; ++I)
#pragma unroll
                            for (int d = 0; d < 3; ++d) u[corner(I, J, K)][d] = sm.us[K ? b1 : b0][d][ty + J][tx + I];
                float2 f[8][3];
                cell_forces2(u, spa, spb, a.cubw, a.cub, eb, f);
#pragma unroll
                for (int J = 0; J < 2; ++J)
#pragma unroll
                    for (int I = 0; I < 2; ++I)
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            sm.fb[I + 2 * J][d][ty][tx] = f[corner(I, J, 0)][d];
                            sm.ft[I + 2 * J][d][ty][tx] = f[corner(I, J, 1)][d];
                        }
            }
            cp_async_wait_all();
            __syncthreads();
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                if (tid + m * NT >= no) continue;
                const int i = oi[m], j = oj[m];
                const int sl = pair_slot(i - 1), sr = pair_slot(i);
                if (kk >= k0) {
                    const long long nidx = 3 * (ocol[m] + poff);
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const float *f3 = reinterpret_cast<const float *>(&sm.fb[3][d][j - 1][0]);
                        const float *f2 = reinterpret_cast<const float *>(&sm.fb[2][d][j - 1][0]);
                        const float *f1 = reinterpret_cast<const float *>(&sm.fb[1][d][j][0]);
                        const float *f0 = reinterpret_cast<const float *>(&sm.fb[0][d][j][0]);
                        const float F = acc[m][d] + f3[sl] + f2[sr] + f1[sl] + f0[sr];
                        const float vn = rfma(fscale, F, rmul(a.keep, vold[m][d]));
                        a.v[nidx + d] = vn;
                        const float *ur = reinterpret_cast<const float *>(&sm.us[b0][d][j][0]);
                        a.u_out[nidx + d] = rfma(a.dt, vn, ur[i <= 8 ? 2 * i : 2 * (i - 8) + 1]);
                    }
                }
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const float *f3 = reinterpret_cast<const float *>(&sm.ft[3][d][j - 1][0]);
                    const float *f2 = reinterpret_cast<const float *>(&sm.ft[2][d][j - 1][0]);
                    const float *f1 = reinterpret_cast<const float *>(&sm.ft[1][d][j][0]);
                    const float *f0 = reinterpret_cast<const float *>(&sm.ft[0][d][j][0]);
                    acc[m][d] = f3[sl] + f2[sr] + f1[sl] + f0[sr];
                }
            }
            __syncthreads();
            const int t = b0;
            b0 = b1;
            b1 = b2;
            b2 = t;
            spa = spa_n;
            spb = spb_n;
        }
    }
}

template <typename T, int CX, int CY>
size_t smem_of(bool stab, int nq) {
    return stab ? mpm_table_offset<CX, CY, T>() + sizeof(float) * 12 * (size_t)nq
                : sizeof(typename MpmSmem<CX, CY>::template S<T>);
}

}  // namespace

int mpm_shape_cx(int shape) { return shape == MPM_32x8 ? 32 : shape == MPM_8x32 ? 8 : 16; }
int mpm_shape_cy(int shape) { return shape == MPM_32x8 ? 8 : shape == MPM_8x32 ? 32 : 16; }

template <typename T, int CX, int CY, bool PAIR, bool STAB>
static cudaError_t set_attr() {
    return cudaFuncSetAttribute(k_mpm_step<T, CX, CY, PAIR, STAB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_of<T, CX, CY>(STAB, MPM_STAB_MAX));
}

template <bool PAIR, bool STAB>
static cudaError_t set_attr_f32() {
    cudaError_t e;
    if ((e = set_attr<float, 16, 16, PAIR, STAB>()) != cudaSuccess) return e;
    if ((e = set_attr<float, 32, 8, PAIR, STAB>()) != cudaSuccess) return e;
    return set_attr<float, 8, 32, PAIR, STAB>();
}

cudaError_t mpm_prepare() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_mpm_step2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sizeof(MpmSmem2))) != cudaSuccess)
        return e;
    if ((e = set_attr_f32<false, false>()) != cudaSuccess || (e = set_attr_f32<false, true>()) != cudaSuccess ||
        (e = set_attr_f32<true, false>()) != cudaSuccess || (e = set_attr_f32<true, true>()) != cudaSuccess ||
        (e = set_attr<double, 16, 16, false, false>()) != cudaSuccess ||
        (e = set_attr<double, 32, 8, false, false>()) != cudaSuccess ||
        (e = set_attr<double, 8, 32, false, false>()) != cudaSuccess)
        return e;
    return cudaSuccess;
}

template <typename T, bool PAIR, bool STAB>
static int per_sm_t(int shape, int nq) {
    int n = 1;
    cudaError_t e;
    if (shape == MPM_32x8)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mpm_step<T, 32, 8, PAIR, STAB>, 256,
                                                          smem_of<T, 32, 8>(STAB, nq));
    else if (shape == MPM_8x32)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mpm_step<T, 8, 32, PAIR, STAB>, 256,
                                                          smem_of<T, 8, 32>(STAB, nq));
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mpm_step<T, 16, 16, PAIR, STAB>, 256,
                                                          smem_of<T, 16, 16>(STAB, nq));
    return (e != cudaSuccess || n < 1) ? 1 : n;
}

template <>
int mpm_per_sm<float>(int shape, int nq) {
    if (shape == MPM_TWO_CELL) {
        int n = 1;
        const cudaError_t e =
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mpm_step2, 128, sizeof(MpmSmem2));
        return (e != cudaSuccess || n < 1) ? 1 : n;
    }
    const int sh = shape % MPM_NSHAPES;
    int a, b;
    if (nq <= MPM_STAB_MAX) {
        a = per_sm_t<float, false, true>(sh, nq);
        b = per_sm_t<float, true, true>(sh, nq);
    } else {
        a = per_sm_t<float, false, false>(sh, nq);
        b = per_sm_t<float, true, false>(sh, nq);
    }
    return a < b ? a : b;
}
template <>
int mpm_per_sm<double>(int shape, int nq) {
    return per_sm_t<double, false, false>(shape % MPM_NSHAPES, nq);
}

// launched with programmatic stream serialisation: the kernel waits for the grid before it
// (griddepcontrol.wait) only after its prologue
template <typename T, int CX, int CY, bool PAIR, bool STAB>
static cudaError_t launch_pdl(const MpmArgs<T> &a, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem_of<T, CX, CY>(STAB, a.nq);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_mpm_step<T, CX, CY, PAIR, STAB>, a);
}
template <typename T, bool PAIR, bool STAB>
static cudaError_t launch_t(const MpmArgs<T> &a, int shape, cudaStream_t s) {
    if (shape == MPM_32x8) return launch_pdl<T, 32, 8, PAIR, STAB>(a, s);
    if (shape == MPM_8x32) return launch_pdl<T, 8, 32, PAIR, STAB>(a, s);
    return launch_pdl<T, 16, 16, PAIR, STAB>(a, s);
}

// shape in 0..2: scalar Hooke; shape + MPM_NSHAPES: paired-FMA Hooke (FP32 only);
// MPM_TWO_CELL: two cells per thread (FP32 only).  FP32 steps of up to MPM_STAB_MAX
// orientations hold the orientation table in shared memory.
template <>
cudaError_t launch_mpm_step<float>(const MpmArgs<float> &a, int shape, cudaStream_t s) {
    const bool stab = a.nq <= MPM_STAB_MAX;
    if (shape == MPM_TWO_CELL) {
        k_mpm_step2<<<a.grid, 128, sizeof(MpmSmem2), s>>>(a);
        return cudaGetLastError();
    }
    if (shape >= MPM_NSHAPES)
        return stab ? launch_t<float, true, true>(a, shape - MPM_NSHAPES, s)
                    : launch_t<float, true, false>(a, shape - MPM_NSHAPES, s);
    return stab ? launch_t<float, false, true>(a, shape, s) : launch_t<float, false, false>(a, shape, s);
}
template <>
cudaError_t launch_mpm_step<double>(const MpmArgs<double> &a, int shape, cudaStream_t s) {
    return launch_t<double, false, false>(a, shape % MPM_NSHAPES, s);
}

}  // namespace hmc
