// Constant-traction zone of the 27 material points around a trial site: the
// elastic part of the trial energy over a zone of half-width one point (Eq. 6;
// the paper's proposed larger zone, Sec. "Conclusions").  The zone is
// re-equilibrated after the site's orientation changes while the forces that
// the rest of the body exerts on the zone's nodes stay at their current values.
// Only the site's stiffness changes and the old zone energy is stationary at the
// current displacement, so the change of the zone's minimum potential energy is
// the rank-6 form
//     dH_e / lambda = 1/2 e0 . dC (I + G dC)^-1 e0,
// e0 = the site's strain, dC = C'(q_new) - C'(q_old), and G = B_p K^+ B_p^T the
// compliance of the zone seen at the site (K: the zone's stiffness with the old
// orientations, B_p: the site's strain-displacement map).
//
// The zone spans 2x2x2 MPM cells and their 3x3x3 nodes (81 DOFs).  K is
// singular only in the six rigid-body modes, which B_p does not see; holding six
// DOFs of three non-collinear nodes outside the site's cell fixed removes them
// without changing G.  G then follows from a block (3x3 per node) Cholesky
// factorisation: the 19 nodes outside the site's cell are eliminated first
// (corners, which create no fill, then edges, then face centres), the site's own
// 8 nodes last, and with B_p^T nonzero only on those, G = Y^T Y for
// Y = L22^-1 B_p^T from the trailing 24x24 factor.  Node coordinates are
// reflected so that the site's cell is always the zone's cell (1,1,1); the
// elimination schedule (which block pairs are structurally nonzero) is then the
// same for every site and is built once on the host.
//
// One warp per trial, taken from the work list that the compaction pass of the
// sweep writes; the zone matrix lives in shared memory; the zone's orientations
// are read from the copy of the spins taken at the start of the half step, and
// accepted trials are XOR-ed into the live spins (the old value is known).
#include <algorithm>
#include <vector>

#include "hmc_device.cuh"

namespace hmc {

namespace {

constexpr int ZS = 81;                       // row stride of the zone matrix (odd: rows in distinct banks)
constexpr int ZK = 6564;                     // 81 x 81 elements rounded up to a multiple of 4
constexpr int ZSCHED_CAP = 1280;             // u16 entries of the elimination schedule
constexpr int ZS_NBOFF = 27, ZS_PROFF = 55;  // schedule header: node order, then the two offset arrays

template <typename T>
struct ZoneCfg;
template <>
struct ZoneCfg<float> {
    static constexpr int WARPS = 4;
};
template <>
struct ZoneCfg<double> {
    static constexpr int WARPS = 2;
};

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }
__host__ __device__ constexpr size_t zone_cta_bytes() { return align16((ZSCHED_CAP + 300) * sizeof(uint16_t)); }
template <typename T>
__host__ __device__ constexpr size_t zone_warp_bytes() {
    return align16((ZK + 144 + 36) * sizeof(T) + 64 + 8);
}
template <typename T>
__host__ __device__ constexpr size_t zone_smem() {
    return zone_cta_bytes() + ZoneCfg<T>::WARPS * zone_warp_bytes<T>();
}

__device__ __forceinline__ float zlog(float x) { return logf(x); }
__device__ __forceinline__ double zlog(double x) { return log(x); }

// Gradient of the trilinear shape function of cell corner (I,J,K) at the point
// of local position (a,b,c) in {0,1}^3 (coordinates 1/4, 3/4 of the edge h = 2).
template <typename T>
__device__ __forceinline__ void corner_grad(int a, int b, int c, int I, int J, int K, T (&g)[3]) {
    const T xa = a ? T(0.75) : T(0.25), xb = b ? T(0.75) : T(0.25), xc = c ? T(0.75) : T(0.25);
    const T Na = I ? xa : T(1) - xa, Nb = J ? xb : T(1) - xb, Nc = K ? xc : T(1) - xc;
    const T sa = I ? T(0.5) : T(-0.5), sb = J ? T(0.5) : T(-0.5), sc = K ? T(0.5) : T(-0.5);
    g[0] = sa * Nb * Nc;
    g[1] = Na * sb * Nc;
    g[2] = Na * Nb * sc;
}

// Row (corner, alpha) of B_p^T: strain (Voigt, engineering shear) per unit
// displacement component alpha of that corner.
template <typename T>
__device__ __forceinline__ void bt_row(const T (&g)[3], int alpha, T (&b)[6]) {
    b[0] = alpha == 0 ? g[0] : T(0);
    b[1] = alpha == 1 ? g[1] : T(0);
    b[2] = alpha == 2 ? g[2] : T(0);
    b[3] = alpha == 1 ? g[2] : alpha == 2 ? g[1] : T(0);
    b[4] = alpha == 0 ? g[2] : alpha == 2 ? g[0] : T(0);
    b[5] = alpha == 0 ? g[1] : alpha == 1 ? g[0] : T(0);
}

template <typename T>
__global__ void __launch_bounds__(32 * ZoneCfg<T>::WARPS) k_zone(ZoneArgs<T> a) {
    constexpr int W = ZoneCfg<T>::WARPS;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    uint16_t *sch = reinterpret_cast<uint16_t *>(smem);
    uint16_t *ep = sch + ZSCHED_CAP;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wb = smem + zone_cta_bytes() + warp * zone_warp_bytes<T>();
    T *Kz = reinterpret_cast<T *>(wb);
    T *Ys = Kz + ZK;          // Y = L22^-1 B_p^T, 24 x 6
    T *Gs = Ys + 144;         // G, 6 x 6
    uint8_t *dmap = reinterpret_cast<uint8_t *>(Gs + 36);   // (zone cell, corner) -> node order
    uint8_t *inv = dmap + 64;                               // order - 19 -> corner of the site's cell

    for (int i = threadIdx.x; i < a.nsched; i += blockDim.x) sch[i] = a.sched[i];
    // element-matrix entry t (upper triangle of the 24 x 24, row-major) -> corners and components
    for (int t = threadIdx.x; t < 300; t += blockDim.x) {
        int e1 = 0, rem = t;
        while (rem >= 24 - e1) {
            rem -= 24 - e1;
            ++e1;
        }
        const int e2 = e1 + rem;
        ep[t] = (uint16_t)((e1 / 3) | ((e1 % 3) << 3) | ((e2 / 3) << 5) | ((e2 % 3) << 8));
    }
    __syncthreads();
    // fixed DOFs: all of node A (order 0), y and z of node B, z of node C
    const int ordB = sch[1], ordC = sch[3];
    const int fB1 = 3 * ordB + 1, fB2 = 3 * ordB + 2, fC2 = 3 * ordC + 2;
    const unsigned n = *a.count;

    for (unsigned e = blockIdx.x * W + warp; e < n; e += gridDim.x * W) {
        const uint4 en = a.work[e];
        const int p = (int)en.x;
        const Replica &R = a.reps[en.y];
        const uint32_t qn = en.z & 0xffffu, q = en.z >> 16, r1 = en.w;
        const int nx = R.nx, ny = R.ny, nz = R.nz;
        const int x = p % nx, yz = p / nx, y = yz % ny, z = yz / ny;
        const int lox = (x - 1) >> 1, loy = (y - 1) >> 1, loz = (z - 1) >> 1;   // lowest zone node (may be -1)
        const int pcx = (x >> 1) - lox, pcy = (y >> 1) - loy, pcz = (z >> 1) - loz;   // site's zone cell

        // the zone's 27 points: orientation (start-of-step copy), position in its cell, zone cell
        uint32_t my_q = 0, my_pos = 0, my_cell = 0;
        if (lane < 27) {
            const int X = x + lane % 3 - 1, Yv = y + (lane / 3) % 3 - 1, Z = z + lane / 9 - 1;
            const int Xw = wrapi(X, nx), Yw = wrapi(Yv, ny), Zw = wrapi(Z, nz);
            const uint4 b = a.snap[R.blk_off + (Xw >> 1) + (long long)R.nbx * ((Yw >> 1) + (long long)R.nby * (Zw >> 1))];
            my_q = spin_of(b, local_slot((Xw & 1) + 2 * (Yw & 1) + 4 * (Zw & 1)));
            my_pos = (Xw & 1) + 2 * (Yw & 1) + 4 * (Zw & 1);
            my_cell = ((X >> 1) - lox) + 2 * ((Yv >> 1) - loy) + 4 * ((Z >> 1) - loz);
        }
        for (int l = lane; l < 64; l += 32) {
            const int c = l >> 3, k = l & 7;
            const int lx = (c & 1) + (k & 1), ly = ((c >> 1) & 1) + ((k >> 1) & 1), lz = (c >> 2) + (k >> 2);
            const int rx = pcx ? lx : 2 - lx, ry = pcy ? ly : 2 - ly, rz = pcz ? lz : 2 - lz;
            const uint8_t o = (uint8_t)sch[rx + 3 * ry + 9 * rz];
            dmap[l] = o;
            if (c == pcx + 2 * pcy + 4 * pcz) inv[o - 19] = (uint8_t)k;
        }
        {
            using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
            V *kv = reinterpret_cast<V *>(Kz);
            const V zero{};
            for (int i = lane; i < (int)(ZK * sizeof(T) / 16); i += 32) kv[i] = zero;
        }
        __syncwarp();
        if (lane < 6) {
            const int d = lane < 3 ? lane : lane == 3 ? fB1 : lane == 4 ? fB2 : fC2;
            Kz[d * ZS + d] = T(1);
        }

        // assembly: K = sum over the zone's points of B^T C' B (element tables per orientation and position)
        for (int s = 0; s < 27; ++s) {
            const uint32_t qs = __shfl_sync(FULL, my_q, s), pos = __shfl_sync(FULL, my_pos, s);
            const uint32_t cell = __shfl_sync(FULL, my_cell, s);
            const T *ke = a.ktab + ((size_t)qs * 8 + pos) * 300;
            const uint8_t *dm = dmap + 8 * cell;
            for (int t = lane; t < 300; t += 32) {
                const uint32_t pr = ep[t];
                const int d1 = 3 * dm[pr & 7] + ((pr >> 3) & 3), d2 = 3 * dm[(pr >> 5) & 7] + (pr >> 8);
                const bool fx = d1 < 3 || d2 < 3 || d1 == fB1 || d1 == fB2 || d1 == fC2 || d2 == fB1 || d2 == fB2 ||
                                d2 == fC2;
                if (fx) continue;
                const int i = max(d1, d2), j = min(d1, d2);
                Kz[i * ZS + j] += __ldg(ke + t);
            }
            __syncwarp();
        }

        // block Cholesky in the static order; a non-positive pivot marks the trial as failed
        bool ok = true;
        for (int k = 0; k < 27; ++k) {
            T *Kk = Kz + 3 * k * ZS + 3 * k;
            const T c00 = Kk[0], c10 = Kk[ZS], c11 = Kk[ZS + 1], c20 = Kk[2 * ZS], c21 = Kk[2 * ZS + 1],
                    c22 = Kk[2 * ZS + 2];
            const T l00 = sqrt(c00), i00 = T(1) / l00;
            const T l10 = c10 * i00, l20 = c20 * i00;
            const T l11 = sqrt(c11 - l10 * l10), i11 = T(1) / l11;
            const T l21 = (c21 - l20 * l10) * i11;
            const T l22 = sqrt(c22 - l20 * l20 - l21 * l21), i22 = T(1) / l22;
            ok = ok && (l00 > T(0)) && (l11 > T(0)) && (l22 > T(0)) && (i00 < T(3.0e38)) && (i11 < T(3.0e38)) &&
                 (i22 < T(3.0e38));
            __syncwarp();
            if (lane == 0) {
                Kk[0] = l00;
                Kk[ZS] = l10;
                Kk[ZS + 1] = l11;
                Kk[2 * ZS] = l20;
                Kk[2 * ZS + 1] = l21;
                Kk[2 * ZS + 2] = l22;
            }
            const int nb0 = sch[ZS_NBOFF + k], nb1 = sch[ZS_NBOFF + k + 1];
            for (int t = nb0 + lane; t < nb1; t += 32) {
                T *B = Kz + 3 * sch[t] * ZS + 3 * k;   // block (I, k): L_Ik = C_Ik L_kk^-T
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    T *row = B + r * ZS;
                    const T x0 = row[0] * i00;
                    const T x1 = (row[1] - x0 * l10) * i11;
                    const T x2 = (row[2] - x0 * l20 - x1 * l21) * i22;
                    row[0] = x0;
                    row[1] = x1;
                    row[2] = x2;
                }
            }
            __syncwarp();
            const int pr0 = sch[ZS_PROFF + k], pr1 = sch[ZS_PROFF + k + 1];
            for (int t = pr0 + lane; t < pr1; t += 32) {
                const int I = sch[t] & 0xff, J = sch[t] >> 8;
                const T *LI = Kz + 3 * I * ZS + 3 * k, *LJ = Kz + 3 * J * ZS + 3 * k;
                T li[3][3], lj[3][3];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        li[r][m] = LI[r * ZS + m];
                        lj[r][m] = LJ[r * ZS + m];
                    }
                T *C = Kz + 3 * I * ZS + 3 * J;
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        if (I != J || c <= r)
                            C[r * ZS + c] -= li[r][0] * lj[c][0] + li[r][1] * lj[c][1] + li[r][2] * lj[c][2];
            }
            __syncwarp();
        }

        // Y = L22^-1 B_p^T on the site's cell (orders 19..26): lane v < 6 takes column v
        const int pa = x & 1, pb = y & 1, pcq = z & 1;
        if (lane < 6) {
            for (int nn = 19; nn < 27; ++nn) {
                const int cr = inv[nn - 19];
                T g[3];
                corner_grad<T>(pa, pb, pcq, cr & 1, (cr >> 1) & 1, cr >> 2, g);
                T rhs[3];
#pragma unroll
                for (int al = 0; al < 3; ++al) {
                    T b[6];
                    bt_row<T>(g, al, b);
                    T v = b[0];
#pragma unroll
                    for (int w = 1; w < 6; ++w)
                        if (lane == w) v = b[w];
                    rhs[al] = v;
                }
                for (int m = 19; m < nn; ++m) {
                    const T *L = Kz + 3 * nn * ZS + 3 * m;
#pragma unroll
                    for (int r = 0; r < 3; ++r)
                        rhs[r] -= L[r * ZS] * Ys[(3 * (m - 19)) * 6 + lane] + L[r * ZS + 1] * Ys[(3 * (m - 19) + 1) * 6 + lane] +
                                  L[r * ZS + 2] * Ys[(3 * (m - 19) + 2) * 6 + lane];
                }
                const T *Ln = Kz + 3 * nn * ZS + 3 * nn;
                const T y0 = rhs[0] / Ln[0];
                const T y1 = (rhs[1] - Ln[ZS] * y0) / Ln[ZS + 1];
                const T y2 = (rhs[2] - Ln[2 * ZS] * y0 - Ln[2 * ZS + 1] * y1) / Ln[2 * ZS + 2];
                Ys[(3 * (nn - 19)) * 6 + lane] = y0;
                Ys[(3 * (nn - 19) + 1) * 6 + lane] = y1;
                Ys[(3 * (nn - 19) + 2) * 6 + lane] = y2;
            }
        }
        __syncwarp();
        if (lane < 21) {
            int v = 0, rem = lane;
            while (rem >= 6 - v) {
                rem -= 6 - v;
                ++v;
            }
            const int w = v + rem;
            T s = T(0);
            for (int rrow = 0; rrow < 24; ++rrow) s += Ys[rrow * 6 + v] * Ys[rrow * 6 + w];
            Gs[6 * v + w] = s;
            Gs[6 * w + v] = s;
        }
        // the site's strain from its cell's nodal displacements: lane = 3 corner + alpha
        T eps[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        if (lane < 24) {
            const int cr = lane / 3, al = lane % 3;
            const int gi = wrapi((x >> 1) + (cr & 1), R.nbx), gj = wrapi((y >> 1) + ((cr >> 1) & 1), R.nby);
            const int gk = wrapi((z >> 1) + (cr >> 2), R.nbz);
            const T uv = a.u[3 * (R.blk_off + gi + (long long)R.nbx * (gj + (long long)R.nby * gk)) + al];
            T g[3];
            corner_grad<T>(pa, pb, pcq, cr & 1, (cr >> 1) & 1, cr >> 2, g);
            T b[6];
            bt_row<T>(g, al, b);
#pragma unroll
            for (int k = 0; k < 6; ++k) eps[k] = b[k] * uv;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) eps[k] += __shfl_xor_sync(FULL, eps[k], o);
        // bond-energy change from the six face neighbours (zone points 12, 14, 10, 16, 4, 22)
        int dE = 0;
        {
            const int nbs[6] = {12, 14, 10, 16, 4, 22};
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                const uint32_t v = __shfl_sync(FULL, my_q, nbs[j]);
                dE += (v == q) - (v == qn);
            }
        }
        __syncwarp();
        ok = __all_sync(FULL, ok);
        if (lane == 0) {
            T eb[6];
            load_ebar<T>(R.st, eb);
            T e0[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) e0[k] = eb[k] + eps[k];
            // dC = C'(q_new) - C'(q_old), symmetric from the 21 stored entries
            T dC[6][6];
            {
                const T *cn = a.ctab + 24 * (size_t)qn, *co = a.ctab + 24 * (size_t)q;
                int t = 0;
#pragma unroll
                for (int i = 0; i < 6; ++i)
#pragma unroll
                    for (int j = i; j < 6; ++j) {
                        const T d = __ldg(cn + t) - __ldg(co + t);
                        dC[i][j] = d;
                        dC[j][i] = d;
                        ++t;
                    }
            }
            // solve (I + G dC) eta = e0 by Gaussian elimination with partial pivoting
            T M[6][7];
#pragma unroll
            for (int i = 0; i < 6; ++i) {
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    T s = i == j ? T(1) : T(0);
#pragma unroll
                    for (int k = 0; k < 6; ++k) s += Gs[6 * i + k] * dC[k][j];
                    M[i][j] = s;
                }
                M[i][6] = e0[i];
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                int piv = c;
                T best = fabs(M[c][c]);
#pragma unroll
                for (int r = c + 1; r < 6; ++r)
                    if (fabs(M[r][c]) > best) {
                        best = fabs(M[r][c]);
                        piv = r;
                    }
                ok = ok && best > T(0);
#pragma unroll
                for (int j = 0; j < 7; ++j) {
                    T tmp = M[c][j];
#pragma unroll
                    for (int r = c + 1; r < 6; ++r)
                        if (r == piv) {
                            M[c][j] = M[r][j];
                            M[r][j] = tmp;
                        }
                }
                const T ip = T(1) / M[c][c];
#pragma unroll
                for (int r = c + 1; r < 6; ++r) {
                    const T f = M[r][c] * ip;
#pragma unroll
                    for (int j = c; j < 7; ++j) M[r][j] -= f * M[c][j];
                }
            }
            T eta[6];
#pragma unroll
            for (int i = 5; i >= 0; --i) {
                T s = M[i][6];
#pragma unroll
                for (int j = i + 1; j < 6; ++j) s -= M[i][j] * eta[j];
                eta[i] = s / M[i][i];
            }
            T f = T(0);
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                T s = T(0);
#pragma unroll
                for (int j = 0; j < 6; ++j) s += dC[i][j] * eta[j];
                f += e0[i] * s;
            }
            const T dHe = (T)R.lam * T(0.5) * f;
            bool acc;
            if (!ok || !(dHe == dHe)) {
                R.st->nonfinite = 1;
                acc = false;
            } else if (dHe == T(0)) {
                acc = dE <= 0 || (unsigned long long)r1 < __ldg(a.thr + dE);
            } else {
                const T H = a.J * (T)dE + dHe;
                const T u01 = ((T)r1 + T(0.5)) * T(2.3283064365386963e-10);
                const T t = a.kT > T(0) ? -a.kT * zlog(u01) : T(0);
                acc = H <= t;
            }
            if (acc) {
                const long long blk =
                    R.blk_off + (x >> 1) + (long long)R.nbx * ((y >> 1) + (long long)R.nby * (z >> 1));
                const int slot = local_slot((x & 1) + 2 * (y & 1) + 4 * (z & 1));
                uint32_t *wp = reinterpret_cast<uint32_t *>(a.spins + blk) + (slot >> 1);
                atomicXor(wp, (q ^ qn) << (16 * (slot & 1)));
                atomicAdd(&R.st->accepted, 1ull);
            }
        }
        __syncwarp();
    }
}

}  // namespace

template <typename T>
size_t zone_smem_bytes() {
    return zone_smem<T>();
}

template <typename T>
int zone_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_zone<T>, 32 * ZoneCfg<T>::WARPS, zone_smem<T>()) !=
        cudaSuccess)
        return 1;
    return std::max(n, 1);
}

cudaError_t zone_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_zone<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)zone_smem<float>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_zone<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)zone_smem<double>());
}

template <typename T>
cudaError_t launch_zone(const ZoneArgs<T> &a, int grid, cudaStream_t s) {
    k_zone<T><<<grid, 32 * ZoneCfg<T>::WARPS, zone_smem<T>(), s>>>(a);
    return cudaGetLastError();
}

template size_t zone_smem_bytes<float>();
template size_t zone_smem_bytes<double>();
template int zone_per_sm<float>();
template int zone_per_sm<double>();
template cudaError_t launch_zone<float>(const ZoneArgs<float> &, int, cudaStream_t);
template cudaError_t launch_zone<double>(const ZoneArgs<double> &, int, cudaStream_t);

// ---- host tables --------------------------------------------------------------

// Elimination schedule of the zone's 27 nodes in the reflected frame (the
// site's cell = nodes with all coordinates in {1,2}).  Layout (uint16):
//   [0, 27)   order of node rx + 3 ry + 9 rz
//   [27, 55)  nb_off[k]: first entry of step k's column blocks (node orders > k)
//   [55, 83)  pr_off[k]: first entry of step k's block updates (I | J << 8, I >= J)
//   then the column-block entries, then the block-update entries.
// Nodes share a block of K when they lie in a common zone cell (Chebyshev
// distance <= 1); the symbolic factorisation adds the fill of each step.
std::vector<uint16_t> zone_schedule() {
    auto co = [](int n, int d) { return d == 0 ? n % 3 : d == 1 ? (n / 3) % 3 : n / 9; };
    auto cls = [&](int n) {
        const int a = co(n, 0), b = co(n, 1), c = co(n, 2);
        if (std::min(a, std::min(b, c)) >= 1) return 3;   // the site's cell
        return (a == 1) + (b == 1) + (c == 1);            // 0 corner, 1 edge, 2 face centre
    };
    std::vector<int> order;
    order.push_back(0);   // node A = (0,0,0): all three DOFs fixed
    for (int n = 1; n < 27; ++n)
        if (cls(n) == 0) order.push_back(n);
    order.push_back(1);   // node B = (1,0,0): y, z fixed
    order.push_back(3);   // node C = (0,1,0): z fixed
    for (int n = 0; n < 27; ++n)
        if (cls(n) == 1 && n != 1 && n != 3) order.push_back(n);
    for (int c = 2; c <= 3; ++c)
        for (int n = 0; n < 27; ++n)
            if (cls(n) == c) order.push_back(n);
    std::vector<uint16_t> t(83, 0);
    for (int i = 0; i < 27; ++i) t[order[i]] = (uint16_t)i;
    bool pat[27][27];
    for (int i = 0; i < 27; ++i)
        for (int j = 0; j < 27; ++j) {
            int dmax = 0;
            for (int d = 0; d < 3; ++d) dmax = std::max(dmax, std::abs(co(order[i], d) - co(order[j], d)));
            pat[i][j] = dmax <= 1;
        }
    std::vector<std::vector<int>> nb(27);
    std::vector<std::vector<uint16_t>> pr(27);
    for (int k = 0; k < 27; ++k) {
        for (int i = k + 1; i < 27; ++i)
            if (pat[i][k]) nb[k].push_back(i);
        for (int I : nb[k])
            for (int J : nb[k])
                if (J <= I) {
                    pr[k].push_back((uint16_t)(I | (J << 8)));
                    pat[I][J] = pat[J][I] = true;
                }
    }
    size_t off = 83;
    for (int k = 0; k <= 27; ++k) {
        t[ZS_NBOFF + k] = (uint16_t)off;
        if (k < 27) off += nb[k].size();
    }
    for (int k = 0; k <= 27; ++k) {
        t[ZS_PROFF + k] = (uint16_t)off;
        if (k < 27) off += pr[k].size();
    }
    for (int k = 0; k < 27; ++k)
        for (int i : nb[k]) t.push_back((uint16_t)i);
    for (int k = 0; k < 27; ++k)
        for (uint16_t v : pr[k]) t.push_back(v);
    if (t.size() > (size_t)ZSCHED_CAP) t.clear();
    return t;
}

// Element stiffness V B^T C'(q) B (V = 1 voxel) of a point at local position
// pos = a + 2b + 4c of its cell, in element DOF order 3 corner + alpha, upper
// triangle row-major (300 values), for every orientation.
void zone_element_tables(const double *Cv, int Q, std::vector<double> &out) {
    out.assign((size_t)Q * 8 * 300, 0.0);
    for (int pos = 0; pos < 8; ++pos) {
        const int a = pos & 1, b = (pos >> 1) & 1, c = pos >> 2;
        double B[6][24] = {};
        for (int cr = 0; cr < 8; ++cr) {
            const int I = cr & 1, J = (cr >> 1) & 1, K = cr >> 2;
            const double xa = a ? 0.75 : 0.25, xb = b ? 0.75 : 0.25, xc = c ? 0.75 : 0.25;
            const double Na = I ? xa : 1 - xa, Nb = J ? xb : 1 - xb, Nc = K ? xc : 1 - xc;
            const double sa = I ? 0.5 : -0.5, sb = J ? 0.5 : -0.5, sc = K ? 0.5 : -0.5;
            const double g0 = sa * Nb * Nc, g1 = Na * sb * Nc, g2 = Na * Nb * sc;
            B[0][3 * cr + 0] = g0; B[4][3 * cr + 0] = g2; B[5][3 * cr + 0] = g1;
            B[1][3 * cr + 1] = g1; B[3][3 * cr + 1] = g2; B[5][3 * cr + 1] = g0;
            B[2][3 * cr + 2] = g2; B[3][3 * cr + 2] = g1; B[4][3 * cr + 2] = g0;
        }
        for (int q = 0; q < Q; ++q) {
            const double *C = Cv + (size_t)q * 36;
            double CB[6][24];
            for (int i = 0; i < 6; ++i)
                for (int e = 0; e < 24; ++e) {
                    double s = 0;
                    for (int k = 0; k < 6; ++k) s += C[6 * i + k] * B[k][e];
                    CB[i][e] = s;
                }
            double *o = &out[((size_t)q * 8 + pos) * 300];
            int t = 0;
            for (int e1 = 0; e1 < 24; ++e1)
                for (int e2 = e1; e2 < 24; ++e2) {
                    double s = 0;
                    for (int i = 0; i < 6; ++i) s += B[i][e1] * CB[i][e2];
                    o[t++] = s;
                }
        }
    }
}

}  // namespace hmc
