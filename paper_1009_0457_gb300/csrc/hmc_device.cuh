// Device helpers of libhmc: the Philox stream, the block/slot layout, and the
// per-cell material-point arithmetic shared by the MPM step and the stress pass.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hmc_internal.h"

namespace hmc {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products with the Weyl key increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                         uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // each 32 x 32 -> 64-bit product as one wide multiply (both halves at once)
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// the same with the round keys given (philox_round_keys): kernels whose key is the same for
// every thread read them from the kernel argument instead of forming them
__device__ __forceinline__ uint4 philox4_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            const uint32_t (&rk)[20]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ rk[2 * r], n2 = hi0 ^ c3 ^ rk[2 * r + 1];
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// ---------------------------------------------------------------------------
// Block layout.  Local corner index L = lx + 2 ly + 4 lz of a voxel inside its
// 2x2x2 block; slot = position of the voxel's uint16 in the block's uint4.
// Red slots 0..3 hold L = 0,3,5,6 and black slots 4..7 hold L = 1,2,4,7, so the
// x, y and z partners of red slot i are black slots i, i^1, i^2 (and back).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int slot_local(int s) {
    return s == 0 ? 0 : s == 1 ? 3 : s == 2 ? 5 : s == 3 ? 6 : s == 4 ? 1 : s == 5 ? 2 : s == 6 ? 4 : 7;
}
__host__ __device__ constexpr int local_slot(int L) {
    return L == 0 ? 0 : L == 3 ? 1 : L == 5 ? 2 : L == 6 ? 3 : L == 1 ? 4 : L == 2 ? 5 : L == 4 ? 6 : 7;
}

__device__ __forceinline__ uint16_t spin_of(const uint4 &b, int slot) {
    const uint32_t w = slot < 2 ? b.x : slot < 4 ? b.y : slot < 6 ? b.z : b.w;
    return (uint16_t)((slot & 1) ? (w >> 16) : (w & 0xffffu));
}
__device__ __forceinline__ uint16_t quad_get(const uint2 &q, int i) {
    const uint32_t w = i < 2 ? q.x : q.y;
    return (uint16_t)((i & 1) ? (w >> 16) : (w & 0xffffu));
}

__device__ __forceinline__ uint32_t udiv(const UDiv &D, uint32_t n) {
    const uint32_t t = __umulhi(D.m, n);
    return (t + ((n - t) >> D.s1)) >> D.s2;
}

// block coordinates of block `blk` of a replica
__device__ __forceinline__ void block_xyz(const Replica &R, int blk, int &bx, int &by, int &bz) {
    const uint32_t rr = udiv(R.divx, (uint32_t)blk), zz = udiv(R.divy, rr);
    bx = blk - (int)rr * R.nbx;
    by = (int)rr - (int)zz * R.nby;
    bz = (int)zz;
}

__host__ __device__ __forceinline__ int wrapi(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

// ---------------------------------------------------------------------------
// One MPM cell = one 2x2x2 block with its eight material points at local
// coordinates 1/4 and 3/4 of the cell edge h = 2 voxels.  Trilinear shape
// functions are separable, so the displacement gradient along x at point
// (a,b,c) depends only on (b,c): differences of the corner displacements along
// x, interpolated with weights 3/4, 1/4 in y and z (and likewise for y, z).
// The constants below fold the 1/h of the gradient into the second stage.
// ---------------------------------------------------------------------------
template <typename T>
struct CellGrad {
    T gx[2][2][3];  // [b][c][d]  d u_d / dx
    T gy[2][2][3];  // [a][c][d]  d u_d / dy
    T gz[2][2][3];  // [a][b][d]  d u_d / dz
};

// corner index of node (I,J,K) of a cell
__host__ __device__ constexpr int corner(int I, int J, int K) { return I + 2 * J + 4 * K; }

template <typename T>
__device__ __forceinline__ void interp2(T d00, T d10, T d01, T d11, T (&o)[2][2]) {
    // d_JK -> sum_J sum_K w_J(b) w_K(c) d_JK / h, with w = 3/4 (same side) or 1/4
    const T e00 = T(0.75) * d00 + T(0.25) * d10;  // b = 0, K = 0
    const T e10 = T(0.25) * d00 + T(0.75) * d10;  // b = 1, K = 0
    const T e01 = T(0.75) * d01 + T(0.25) * d11;  // b = 0, K = 1
    const T e11 = T(0.25) * d01 + T(0.75) * d11;  // b = 1, K = 1
    o[0][0] = T(0.375) * e00 + T(0.125) * e01;
    o[0][1] = T(0.125) * e00 + T(0.375) * e01;
    o[1][0] = T(0.375) * e10 + T(0.125) * e11;
    o[1][1] = T(0.125) * e10 + T(0.375) * e11;
}

template <typename T>
__device__ __forceinline__ void cell_gradients(const T (&u)[8][3], CellGrad<T> &g) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        T o[2][2];
        // x differences indexed (J,K)
        interp2<T>(u[corner(1, 0, 0)][d] - u[corner(0, 0, 0)][d], u[corner(1, 1, 0)][d] - u[corner(0, 1, 0)][d],
                   u[corner(1, 0, 1)][d] - u[corner(0, 0, 1)][d], u[corner(1, 1, 1)][d] - u[corner(0, 1, 1)][d], o);
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) g.gx[b][c][d] = o[b][c];
        // y differences indexed (I,K)
        interp2<T>(u[corner(0, 1, 0)][d] - u[corner(0, 0, 0)][d], u[corner(1, 1, 0)][d] - u[corner(1, 0, 0)][d],
                   u[corner(0, 1, 1)][d] - u[corner(0, 0, 1)][d], u[corner(1, 1, 1)][d] - u[corner(1, 0, 1)][d], o);
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int c = 0; c < 2; ++c) g.gy[a][c][d] = o[a][c];
        // z differences indexed (I,J)
        interp2<T>(u[corner(0, 0, 1)][d] - u[corner(0, 0, 0)][d], u[corner(1, 0, 1)][d] - u[corner(1, 0, 0)][d],
                   u[corner(0, 1, 1)][d] - u[corner(0, 1, 0)][d], u[corner(1, 1, 1)][d] - u[corner(1, 1, 0)][d], o);
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) g.gz[a][b][d] = o[a][b];
    }
}

// Strain (Voigt, engineering shear) of point (a,b,c) of the cell.
template <typename T>
__device__ __forceinline__ void point_strain(const CellGrad<T> &g, const T (&eb)[6], int a, int b, int c,
                                             T (&e)[6]) {
    // G[d][k] = d u_d / d x_k
    e[0] = eb[0] + g.gx[b][c][0];
    e[1] = eb[1] + g.gy[a][c][1];
    e[2] = eb[2] + g.gz[a][b][2];
    e[3] = eb[3] + (g.gz[a][b][1] + g.gy[a][c][2]);
    e[4] = eb[4] + (g.gz[a][b][0] + g.gx[b][c][2]);
    e[5] = eb[5] + (g.gy[a][c][0] + g.gx[b][c][1]);
}

template <typename T>
struct Row24;
template <>
struct Row24<float> {
    float v[24];
    __device__ __forceinline__ void load(const float *p) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const float4 t = __ldg(q + i);
            v[4 * i] = t.x;
            v[4 * i + 1] = t.y;
            v[4 * i + 2] = t.z;
            v[4 * i + 3] = t.w;
        }
    }
};
template <>
struct Row24<double> {
    double v[24];
    __device__ __forceinline__ void load(const double *p) {
        const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
        for (int i = 0; i < 11; ++i) {
            const double2 t = __ldg(q + i);
            v[2 * i] = t.x;
            v[2 * i + 1] = t.y;
        }
    }
};

// Explicitly rounded product and fused multiply-add, so that every kernel and
// variant evaluates a dot product in the same order with the same roundings.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// Row i of sigma = C e: C_i0 e0, then C_ij e_j added by fused multiply-adds in
// j order (the order of the paired-FMA variant of the MPM step, which is
// therefore bit-identical).
template <typename T>
__device__ __forceinline__ T hooke_row(T c0, T c1, T c2, T c3, T c4, T c5, const T (&e)[6]) {
    T s = rmul(c0, e[0]);
    s = rfma(c1, e[1], s);
    s = rfma(c2, e[2], s);
    s = rfma(c3, e[3], s);
    s = rfma(c4, e[4], s);
    return rfma(c5, e[5], s);
}

// sigma = C e with the 21 upper-triangle entries c00 c01 .. c05 c11 .. c55.
template <typename T>
__device__ __forceinline__ void hooke21(const T *c, const T (&e)[6], T (&s)[6]) {
    s[0] = hooke_row<T>(c[0], c[1], c[2], c[3], c[4], c[5], e);
    s[1] = hooke_row<T>(c[1], c[6], c[7], c[8], c[9], c[10], e);
    s[2] = hooke_row<T>(c[2], c[7], c[11], c[12], c[13], c[14], e);
    s[3] = hooke_row<T>(c[3], c[8], c[12], c[15], c[16], c[17], e);
    s[4] = hooke_row<T>(c[4], c[9], c[13], c[16], c[18], c[19], e);
    s[5] = hooke_row<T>(c[5], c[10], c[14], c[17], c[19], c[20], e);
}

template <typename T>
__device__ __forceinline__ void load_ebar(const DevState *st, T (&e)[6]);
template <>
__device__ __forceinline__ void load_ebar<float>(const DevState *st, float (&e)[6]) {
#pragma unroll
    for (int i = 0; i < 6; ++i) e[i] = st->ebar_f[i];
}
template <>
__device__ __forceinline__ void load_ebar<double>(const DevState *st, double (&e)[6]) {
#pragma unroll
    for (int i = 0; i < 6; ++i) e[i] = st->ebar[i];
}

}  // namespace hmc
