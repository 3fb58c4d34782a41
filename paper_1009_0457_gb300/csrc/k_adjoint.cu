// Kernels of the hand-written adjoint of the explicit MPM stress solve.
//
// Forward map (spins frozen, theta = (C11, C12, C44, Ebar_1..6)):
//   f^n = F(u^n; theta) = -sum_p V B_p^T C'_p (Ebar + B_p u^n)
//   v^{n+1} = kappa v^n + c f^n,  u^{n+1} = u^n + dt v^{n+1}   (kappa = 1 - damping, c = dt/m)
// outputs W = sum_p w_p and the field w_p = 1/2 eps_p.C'_p.eps_p at u^T.
// For L = gW W + sum_p g_p w_p (alpha_p = gW + g_p) the reverse sweep is
//   ubar^T = sum_p alpha_p B_p^T C'_p eps_p,   lambda^T = dt ubar^T
//   theta_bar += -c [ epsbar_p . R_i . eps_p^n , (C'_p epsbar_p)_k ] summed over p,  epsbar_p = B_p lambda^{n+1}
//   ubar^n = ubar^{n+1} + c F(lambda^{n+1}; Ebar = 0)      (the forward MPM kernel with kappa = 1)
//   lambda^n = kappa lambda^{n+1} + dt ubar^n
// plus the terminal terms sum_p alpha_p [1/2 eps.R_i.eps, (C' eps)_k].  R_i are
// the rotated basis tensors with C' = C11 R_1 + C12 R_2 + C44 R_3.
//
// These kernels: the per-step parameter terms (added to per-CTA partials that
// are reduced once per reverse sweep), the terminal pass (field w, W,
// alpha-weighted nodal vector through a per-cell buffer and a node gather,
// terminal parameter terms), the lambda update, and the fixed-order FP64
// reduction of per-CTA partials.  Single replica; one thread per cell.
#include "hmc_device.cuh"
#include "hmc_adjoint.h"

namespace hmc {

namespace {

template <typename T>
__device__ __forceinline__ void load_corners(const T *__restrict__ u, int bx, int by, int bz, int nbx, int nby,
                                             int nbz, T (&c)[8][3]) {
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
                for (int d = 0; d < 3; ++d) c[corner(I, J, K)][d] = __ldg(u + n + d);
            }
}

template <typename T>
__device__ __forceinline__ T quad21(const T *c, const T (&a)[6], const T (&b)[6]) {
    // a . C . b with the 21 upper-triangle entries of a symmetric 6x6 C
    T s[6];
    hooke21<T>(c, b, s);
    return a[0] * s[0] + a[1] * s[1] + a[2] * s[2] + a[3] * s[3] + a[4] * s[4] + a[5] * s[5];
}

// Error-free sum of two floats (Knuth's TwoSum): a + b = s + e exactly.
struct TwoSumF {
    float hi, lo;
    __device__ __forceinline__ void add(float x) {
        const float s = hi + x;
        const float bb = s - hi;
        const float e = (hi - (s - bb)) + (x - bb);
        hi = s;
        lo += e;
    }
};

// Per-thread accumulators of NV reduced quantities: FP32 values are summed as
// TwoSum pairs (no FP64 arithmetic per point or per cell), FP64 values plainly.
template <typename T, int NV>
struct AdjAcc;
template <int NV>
struct AdjAcc<float, NV> {
    TwoSumF v[NV];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i].hi = v[i].lo = 0.f;
    }
    __device__ __forceinline__ void add(int i, float x) { v[i].add(x); }
    __device__ __forceinline__ void warp_reduce() {
#pragma unroll
        for (int off = 16; off; off >>= 1)
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                const float hi = __shfl_down_sync(0xffffffffu, v[i].hi, off);
                const float lo = __shfl_down_sync(0xffffffffu, v[i].lo, off);
                v[i].add(hi);
                v[i].lo += lo;
            }
    }
    __device__ __forceinline__ double get(int i) const { return (double)v[i].hi + (double)v[i].lo; }
};
template <int NV>
struct AdjAcc<double, NV> {
    double v[NV];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] = 0.0;
    }
    __device__ __forceinline__ void add(int i, double x) { v[i] += x; }
    __device__ __forceinline__ void warp_reduce() {
#pragma unroll
        for (int off = 16; off; off >>= 1)
#pragma unroll
            for (int i = 0; i < NV; ++i) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
    }
    __device__ __forceinline__ double get(int i) const { return v[i]; }
};

// Sum the NV values of every thread into one FP64 partial per CTA, stored, or
// added to the CTA's partial (accumulate: the reverse sweep sums its steps per CTA
// and reduces across CTAs once).
template <typename T, int NV>
__device__ __forceinline__ void cta_partials(AdjAcc<T, NV> &acc, double *partials, bool accumulate) {
    __shared__ double red[8][NV];
    acc.warp_reduce();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int i = 0; i < NV; ++i) red[warp][i] = acc.get(i);
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
        double *p = partials + NV * (long long)blockIdx.x + threadIdx.x;
        *p = accumulate ? *p + s : s;
    }
}

// The basis quadratic forms of a rotated cubic crystal from the crystal-axis
// projections p_m(x) = a_m.x.a_m (x a strain, engineering shear):
//   x.R_1.y = P,  x.R_2.y = tr x tr y - P,  x.R_3.y = 2 (x:y - P),  P = sum_m p_m(x) p_m(y),
// since R_1 holds the crystal-frame normal-normal diagonal, R_2 its off-diagonal
// and R_3 the engineering-shear diagonal.  w holds the Voigt weights of the three
// axes for tensor-shear components, so the shear strains enter halved.
template <typename T>
__device__ __forceinline__ void basis_forms(const T (&w)[18], const T (&x)[6], const T (&y)[6], T (&r)[3]) {
    const T xh[6] = {x[0], x[1], x[2], T(0.5) * x[3], T(0.5) * x[4], T(0.5) * x[5]};
    const T yh[6] = {y[0], y[1], y[2], T(0.5) * y[3], T(0.5) * y[4], T(0.5) * y[5]};
    T P = T(0);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        T px = T(0), py = T(0);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            px += w[6 * m + k] * xh[k];
            py += w[6 * m + k] * yh[k];
        }
        P += px * py;
    }
    const T tr = (x[0] + x[1] + x[2]) * (y[0] + y[1] + y[2]);
    const T dd = x[0] * y[0] + x[1] * y[1] + x[2] * y[2] + x[3] * yh[3] + x[4] * yh[4] + x[5] * yh[5];
    r[0] = P;
    r[1] = tr - P;
    r[2] = T(2) * (dd - P);
}

template <typename T>
__device__ __forceinline__ void load_row(const T *__restrict__ p, int n, T *out) {
#pragma unroll
    for (int k = 0; k < n; ++k) out[k] = __ldg(p + k);
}

// One reverse step's parameter terms: per point epsbar.R_i.eps (i = 1..3) and
// C' epsbar (6); a cell's eight points are summed plainly, cells by the
// accumulator, and the CTA's sums are added to its partials.  The axis weights and
// the stiffness row are loaded when the orientation changes from one point to the next.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_adj_params(AdjArgs<T> a, const T *__restrict__ lam,
                                                    const T *__restrict__ u) {
    AdjAcc<T, 9> acc;
    acc.zero();
    const int blk = blockIdx.x * blockDim.x + threadIdx.x;
    if (blk < a.nblk) {
        const int bx = blk % a.nbx, r = blk / a.nbx;
        const int by = r % a.nby, bz = r / a.nby;
        T cl[8][3], cu[8][3];
        load_corners<T>(lam, bx, by, bz, a.nbx, a.nby, a.nbz, cl);
        load_corners<T>(u, bx, by, bz, a.nbx, a.nby, a.nbz, cu);
        CellGrad<T> gl, gu;
        cell_gradients<T>(cl, gl);
        cell_gradients<T>(cu, gu);
        const uint4 sp = __ldg(a.spins + blk);
        const T zero[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        T csum[9] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
        T w[18];
        Row24<T> crow;
        uint32_t qprev = 0xffffffffu;
#pragma unroll
        for (int L = 0; L < 8; ++L) {
            const int x = L & 1, y = (L >> 1) & 1, z = L >> 2;
            T eb[6], e[6], s[6], rf[3];
            point_strain<T>(gl, zero, x, y, z, eb);
            point_strain<T>(gu, a.ebar, x, y, z, e);
            const uint32_t q = spin_of(sp, local_slot(L));
            if (q != qprev) {
                load_row<T>(a.wtab + 20ll * q, 18, w);
                crow.load(a.ctab + 24ll * q);
                qprev = q;
            }
            basis_forms<T>(w, eb, e, rf);
#pragma unroll
            for (int i = 0; i < 3; ++i) csum[i] += rf[i];
            hooke21<T>(crow.v, eb, s);
#pragma unroll
            for (int k = 0; k < 6; ++k) csum[3 + k] += s[k];
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) acc.add(i, csum[i]);
    }
    cta_partials<T, 9>(acc, a.partials, true);
}

// Terminal pass at u^T: field w (natural order), per-CTA partials of
// [W, sum alpha 1/2 eps.R_i.eps, sum alpha C' eps], and each cell's eight
// corner contributions of sum_p alpha_p B_p^T sigma_p.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_terminal(AdjArgs<T> a, const T *__restrict__ u,
                                                      const T *__restrict__ g, T gW, T *__restrict__ w,
                                                      T *__restrict__ fcell) {
    AdjAcc<T, 10> acc;
    acc.zero();
    const int blk = blockIdx.x * blockDim.x + threadIdx.x;
    if (blk < a.nblk) {
        const int bx = blk % a.nbx, r = blk / a.nbx;
        const int by = r % a.nby, bz = r / a.nby;
        T csum[10] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
        T cu[8][3];
        load_corners<T>(u, bx, by, bz, a.nbx, a.nby, a.nbz, cu);
        CellGrad<T> gu;
        cell_gradients<T>(cu, gu);
        const uint4 sp = __ldg(a.spins + blk);
        T tx[2][2][3], ty[2][2][3], tz[2][2][3];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int d = 0; d < 3; ++d) tx[i][j][d] = ty[i][j][d] = tz[i][j][d] = T(0);
#pragma unroll
        for (int L = 0; L < 8; ++L) {
            const int x = L & 1, y = (L >> 1) & 1, z = L >> 2;
            T e[6], s[6];
            point_strain<T>(gu, a.ebar, x, y, z, e);
            const uint32_t q = spin_of(sp, local_slot(L));
            hooke21<T>(a.ctab + 24ll * q, e, s);
            const long long p = (2 * bx + x) + (long long)a.nx * ((2 * by + y) + (long long)a.ny * (2 * bz + z));
            const T wp = T(0.5) * (s[0] * e[0] + s[1] * e[1] + s[2] * e[2] + s[3] * e[3] + s[4] * e[4] + s[5] * e[5]);
            if (w) w[p] = wp;
            const T al = gW + (g ? g[p] : T(0));
            csum[0] += wp;
            const T *rq = a.rtab + 72ll * q;
#pragma unroll
            for (int i = 0; i < 3; ++i) csum[1 + i] += al * T(0.5) * quad21<T>(rq + 24 * i, e, e);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                csum[4 + k] += al * s[k];
                s[k] *= al;
            }
            tx[y][z][0] += s[0]; tx[y][z][1] += s[5]; tx[y][z][2] += s[4];
            ty[x][z][0] += s[5]; ty[x][z][1] += s[1]; ty[x][z][2] += s[3];
            tz[x][y][0] += s[4]; tz[x][y][1] += s[3]; tz[x][y][2] += s[2];
        }
        // sum_p B_p^T (alpha sigma)_p at the 8 corners: (V/h) [(2I-1) X + (2J-1) Y + (2K-1) Z]
        T *fc = fcell + 24ll * blk;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            T X[2][2], Y[2][2], Z[2][2];
            interp2<T>(tx[0][0][d], tx[1][0][d], tx[0][1][d], tx[1][1][d], X);
            interp2<T>(ty[0][0][d], ty[1][0][d], ty[0][1][d], ty[1][1][d], Y);
            interp2<T>(tz[0][0][d], tz[1][0][d], tz[0][1][d], tz[1][1][d], Z);
#pragma unroll
            for (int K = 0; K < 2; ++K)
#pragma unroll
                for (int J = 0; J < 2; ++J)
#pragma unroll
                    for (int I = 0; I < 2; ++I) {
                        const T fx = I ? X[J][K] : -X[J][K];
                        const T fy = J ? Y[I][K] : -Y[I][K];
                        const T fz = K ? Z[I][J] : -Z[I][J];
                        fc[3 * corner(I, J, K) + d] = fx + fy + fz;
                    }
        }
#pragma unroll
        for (int i = 0; i < 10; ++i) acc.add(i, csum[i]);
    }
    cta_partials<T, 10>(acc, a.partials, false);
}

// Node gather of the per-cell corner contributions (fixed order): out = scale * sum.
template <typename T>
__global__ void k_adj_gather(AdjArgs<T> a, const T *__restrict__ fcell, T scale, T *__restrict__ out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= a.nblk) return;
    const int i = n % a.nbx, r = n / a.nbx;
    const int j = r % a.nby, k = r / a.nby;
    T s[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int K = 0; K < 2; ++K)
#pragma unroll
        for (int J = 0; J < 2; ++J)
#pragma unroll
            for (int I = 0; I < 2; ++I) {
                // the cell that sees this node as corner (I, J, K)
                const int ci = i - I < 0 ? a.nbx - 1 : i - I, cj = j - J < 0 ? a.nby - 1 : j - J;
                const int ck = k - K < 0 ? a.nbz - 1 : k - K;
                const T *fc = fcell + 24ll * (ci + a.nbx * (cj + a.nby * ck)) + 3 * corner(I, J, K);
#pragma unroll
                for (int d = 0; d < 3; ++d) s[d] += fc[d];
            }
#pragma unroll
    for (int d = 0; d < 3; ++d) out[3ll * n + d] = scale * s[d];
}

// lambda <- x - damping * lambda (elementwise over 3 * nnodes values).
template <typename T>
__global__ void k_adj_lambda(long long n, const T *__restrict__ x, T damping, T *__restrict__ lam) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) lam[i] = x[i] - damping * lam[i];
}

// out[i] += scale * sum over CTAs of partials[., i] (fixed order), one CTA.
__global__ void k_adj_reduce(const double *partials, int nparts, int nv, int stride, double scale, double *out) {
    __shared__ double red[256];
    for (int i = 0; i < nv; ++i) {
        double s = 0.0;
        for (int p = threadIdx.x; p < nparts; p += 256) s += partials[(long long)stride * p + i];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = 128; w; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[i] += scale * red[0];
        __syncthreads();
    }
}

}  // namespace

template <typename T>
cudaError_t launch_adj_params(const AdjArgs<T> &a, const T *lam, const T *u, cudaStream_t s) {
    k_adj_params<T><<<(a.nblk + 255) / 256, 256, 0, s>>>(a, lam, u);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_adj_terminal(const AdjArgs<T> &a, const T *u, const T *g, T gW, T *w, T *fcell, cudaStream_t s) {
    k_adj_terminal<T><<<(a.nblk + 255) / 256, 256, 0, s>>>(a, u, g, gW, w, fcell);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_adj_gather(const AdjArgs<T> &a, const T *fcell, T scale, T *out, cudaStream_t s) {
    k_adj_gather<T><<<(a.nblk + 255) / 256, 256, 0, s>>>(a, fcell, scale, out);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_adj_lambda(long long n, const T *x, T damping, T *lam, cudaStream_t s) {
    k_adj_lambda<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, x, damping, lam);
    return cudaGetLastError();
}
cudaError_t launch_adj_reduce(const double *partials, int nparts, int nv, int stride, double scale, double *out,
                              cudaStream_t s) {
    k_adj_reduce<<<1, 256, 0, s>>>(partials, nparts, nv, stride, scale, out);
    return cudaGetLastError();
}

#define HMC_ADJ_INST(T)                                                                                          \
    template cudaError_t launch_adj_params<T>(const AdjArgs<T> &, const T *, const T *, cudaStream_t);         \
    template cudaError_t launch_adj_terminal<T>(const AdjArgs<T> &, const T *, const T *, T, T *, T *,         \
                                                cudaStream_t);                                                \
    template cudaError_t launch_adj_gather<T>(const AdjArgs<T> &, const T *, T, T *, cudaStream_t);            \
    template cudaError_t launch_adj_lambda<T>(long long, const T *, T, T *, cudaStream_t);
HMC_ADJ_INST(float)
HMC_ADJ_INST(double)

}  // namespace hmc
