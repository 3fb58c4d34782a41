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
// orientations, B_p: the site's strain-displacement map).  With K' = K + B_p^T dC B_p,
// the zone's stiffness with the site's new orientation, the Sherman-Morrison-Woodbury
// identity turns this into
//     dH_e / lambda = 1/2 e0 . dC e0 - 1/2 f . K'^+ f,    f = B_p^T dC e0,
// the energy of the stiffness change at the current strain less what the zone
// recovers by relaxing under the force f that the change exerts on the site's nodes.
//
// The zone spans 2x2x2 MPM cells and their 3x3x3 nodes (81 DOFs).  K' is
// singular only in the six rigid-body modes, which f does not load (B_p sees no
// rigid motion); holding six DOFs of three non-collinear nodes outside the site's
// cell fixed removes them without changing f . K'^+ f.  That form follows from a
// block (3x3 per node) Cholesky elimination of K' bordered by f: one pseudo-node
// (order 27) carries f in the first row of its blocks, nonzero only on the site's
// own 8 nodes.  The 19 nodes outside the site's cell are eliminated first (corners,
// which create no fill, then edges and face centres in the order that needs the
// fewest block updates), the site's 8 nodes next, and the pseudo-node never:
// eliminating all 27 real nodes leaves -f . K'^+ f in the first entry of the
// pseudo-node's diagonal block (the Schur complement of K' in the bordered matrix).
// Node coordinates are reflected so that the site's cell is always the zone's cell
// (1,1,1); the elimination schedule (which block pairs are structurally nonzero) is
// then the same for every site and is built once on the host.
//
// One warp per trial, taken from the work list that the compaction pass of the
// sweep writes; the zone matrix lives in shared memory; the zone's orientations
// are read from the copy of the spins taken at the start of the half step, and
// accepted trials are XOR-ed into the live spins (the old value is known).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "hmc_device.cuh"

namespace hmc {

namespace {

// Schedule table (uint16, built by zone_schedule), orders 0..26 the real nodes and 27 the
// pseudo-node of f (ZN = 28 orders):
//   [0, 27)        elimination order of reflected node rx + 3 ry + 9 rz
//   [27]           number of update rounds (the first six are the outer corners' steps 1..6)
//   [83, 110)      slot of the diagonal block of order k
//   [110, 894)     slot of block (I, J), I >= J, of ZN x ZN in the filled pattern (0xffff: zero)
//   [896, ...)     per round and lane: the slots of the lane's update -- target (I, J),
//                  column blocks (I, k) and (J, k), diagonal block (k, k) -- or 0xffff (no update)
constexpr int ZN = 28;
constexpr int ZS_NROUND = 27, ZS_DIAG = 83, ZS_BIDX = 110, ZS_HDR = ZS_BIDX + ZN * ZN;
constexpr int ZS_RND = (ZS_HDR + 3) & ~3;   // 8-byte aligned rounds of 32 x 4 entries
constexpr int ZSCHED_CAP = 5184;
constexpr int ZSLOT_CAP = 218;   // 3x3 blocks of the filled lower triangle (217 for this pattern) + the unused slot
constexpr int ZBLK = 12;         // a block: 3 rows of 4 values (the 4th pads a row to 16 B)
constexpr int ZROW = 320;        // an element matrix's 300 upper-triangle entries, padded to 10 x 32
constexpr int ZTRASH = (ZSLOT_CAP - 1) * ZBLK;   // an unused slot: target of the scatter's padding

template <typename T>
struct ZoneCfg;
template <>
struct ZoneCfg<float> {
    static constexpr int WARPS = 8;
};
template <>
struct ZoneCfg<double> {
    static constexpr int WARPS = 4;
};

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }
__host__ __device__ constexpr size_t zone_sched_bytes() { return align16(ZSCHED_CAP * sizeof(uint16_t)); }
// + per reflection of the site's cell: the zone points grouped by zone cell (32 bytes, 27
// used) and the end of each cell's group (8 bytes)
__host__ __device__ constexpr size_t zone_cta_bytes() { return zone_sched_bytes() + 8 * 32 + 8 * 8; }
template <typename T>
__host__ __device__ constexpr size_t zone_warp_bytes() {
    return align16((ZSLOT_CAP * ZBLK + 36) * sizeof(T));
}

// Zone offsets (-1, 0 or 1) along one axis of the points in zone cell bit cb when the site's
// own cell is cell pc along that axis: the site's cell (pc; 1 in the zone when the
// coordinate is even) holds offsets {0, +1} or {-1, 0}, the other cell the rest.
__device__ __forceinline__ void zone_cell_span(int cb, int pc, int &lo, int &hi) {
    lo = cb ? (pc ? 0 : 1) : -1;
    hi = cb ? 1 : (pc ? -1 : 0);
}
template <typename T>
__host__ __device__ constexpr size_t zone_smem() {
    return zone_cta_bytes() + ZoneCfg<T>::WARPS * zone_warp_bytes<T>();
}

__device__ __forceinline__ float zrsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double zrsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float zlog(float x) { return logf(x); }
__device__ __forceinline__ double zlog(double x) { return log(x); }

// element-row loads: read once per point, mostly L2 hits, and not kept in L1, so that L1
// holds the scatter-place table that every trial reads
__device__ __forceinline__ float ldg_stream(const float *p) {
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double ldg_stream(const double *p) {
    double v;
    asm volatile("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void ld4(const float *p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double *p, const double (&v)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

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

// Component v of row (corner, alpha) of B_p^T: strain (Voigt, engineering
// shear) per unit displacement component alpha of that corner.
template <typename T>
__device__ __forceinline__ T bt_entry(const T (&g)[3], int alpha, int v) {
    switch (v) {
        case 0: return alpha == 0 ? g[0] : T(0);
        case 1: return alpha == 1 ? g[1] : T(0);
        case 2: return alpha == 2 ? g[2] : T(0);
        case 3: return alpha == 1 ? g[2] : alpha == 2 ? g[1] : T(0);
        case 4: return alpha == 0 ? g[2] : alpha == 2 ? g[0] : T(0);
        default: return alpha == 0 ? g[1] : alpha == 1 ? g[0] : T(0);
    }
}

template <typename T>
__global__ void __launch_bounds__(32 * ZoneCfg<T>::WARPS, 2) k_zone(ZoneArgs<T> a) {
    constexpr int W = ZoneCfg<T>::WARPS;
    constexpr int NJ = 10;   // element-matrix entries per lane: t = lane + 32 j < 300
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    uint16_t *sch = reinterpret_cast<uint16_t *>(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wb = smem + zone_cta_bytes() + warp * zone_warp_bytes<T>();
    T *Kb = reinterpret_cast<T *>(wb);                       // block slots of the bordered zone matrix
    T *dCs = Kb + ZSLOT_CAP * ZBLK;                          // C'(q_new) - C'(q_old), 6 x 6
    uint8_t *plist_all = smem + zone_sched_bytes();        // [reflection][32]: points grouped by zone cell
    uint8_t *cend_all = plist_all + 8 * 32;                // [reflection][8]: end of each cell's group

    for (int i = threadIdx.x; i < a.nsched; i += blockDim.x) sch[i] = a.sched[i];
    // the zone's points grouped by zone cell, for each reflection rf (thread 8 rf + cell)
    if (threadIdx.x < 64) {
        const int rf = threadIdx.x >> 3, cell = threadIdx.x & 7;
        const int px = rf & 1, py = (rf >> 1) & 1, pz = rf >> 2;
        int w = 0, x0 = 0, x1 = 0, y0 = 0, y1 = 0, z0 = 0, z1 = 0;
        for (int c = 0; c <= cell; ++c) {
            zone_cell_span(c & 1, px, x0, x1);
            zone_cell_span((c >> 1) & 1, py, y0, y1);
            zone_cell_span(c >> 2, pz, z0, z1);
            if (c < cell) w += (x1 - x0 + 1) * (y1 - y0 + 1) * (z1 - z0 + 1);
        }
        for (int dz = z0; dz <= z1; ++dz)
            for (int dy = y0; dy <= y1; ++dy)
                for (int dx = x0; dx <= x1; ++dx)
                    plist_all[32 * rf + w++] = (uint8_t)((dx + 1) + 3 * (dy + 1) + 9 * (dz + 1));
        cend_all[8 * rf + cell] = (uint8_t)w;
    }
    __syncthreads();
    // fixed DOFs: all of node A (order 0), y and z of node B, z of node C
    const int ordB = sch[1], ordC = sch[3];
    const unsigned n = *a.count;

    // each warp's next work item is read one trial ahead
    const unsigned stride = gridDim.x * W;
    uint4 en_next = make_uint4(0, 0, 0, 0);
    if (blockIdx.x * W + warp < n) en_next = a.work[blockIdx.x * W + warp];
    for (unsigned e = blockIdx.x * W + warp; e < n; e += stride) {
        const uint4 en = en_next;
        if (e + stride < n) en_next = a.work[e + stride];
        const uint32_t p = en.x;   // site index: below 2^32, possibly above 2^31
        const Replica &R = a.reps[en.y];
        const uint32_t qn = en.z & 0xffffu, q = en.z >> 16, r1 = en.w;
        const int nx = R.nx, ny = R.ny, nz = R.nz;
        const uint32_t yz = p / (uint32_t)nx;
        const int x = (int)(p - yz * (uint32_t)nx), y = (int)(yz % (uint32_t)ny), z = (int)(yz / (uint32_t)ny);
        const int lox = (x - 1) >> 1, loy = (y - 1) >> 1, loz = (z - 1) >> 1;   // lowest zone node (may be -1)
        const int pcx = (x >> 1) - lox, pcy = (y >> 1) - loy, pcz = (z >> 1) - loz;   // site's zone cell
        const int refl = pcx + 2 * pcy + 4 * pcz;                                      // its reflection

        // the zone's 27 points: orientation (start-of-step copy) and position in its cell; the
        // assembly takes the site's (zone point 13) stiffness with its new orientation
        uint32_t my_q = 0, my_pos = 0;
        if (lane < 27) {
            const int Xw = wrapi(x + lane % 3 - 1, nx), Yw = wrapi(y + (lane / 3) % 3 - 1, ny);
            const int Zw = wrapi(z + lane / 9 - 1, nz);
            const uint4 b = a.snap[R.blk_off + (Xw >> 1) + (long long)R.nbx * ((Yw >> 1) + (long long)R.nby * (Zw >> 1))];
            my_pos = (Xw & 1) + 2 * (Yw & 1) + 4 * (Zw & 1);
            my_q = spin_of(b, local_slot(my_pos));
        }
        const uint32_t asm_q = lane == 13 ? qn : my_q;
        // inputs of the decision that do not depend on the zone matrix, requested now so that
        // their latency passes during the assembly: the site cell's nodal displacement component
        // of lane 3 corner + alpha (lane < 24), and the two stiffness entries whose difference is
        // entry lane of C'(q_new) - C'(q_old) (lane < 21)
        T uv = T(0), c_new = T(0), c_old = T(0);
        if (lane < 24) {
            const int cr = lane / 3, al = lane % 3;
            const int gi = wrapi((x >> 1) + (cr & 1), R.nbx), gj = wrapi((y >> 1) + ((cr >> 1) & 1), R.nby);
            const int gk = wrapi((z >> 1) + (cr >> 2), R.nbz);
            uv = a.u[3 * (R.blk_off + gi + (long long)R.nbx * (gj + (long long)R.nby * gk)) + al];
        }
        if (lane < 21) {
            c_new = __ldg(a.ctab + 24 * (size_t)qn + lane);
            c_old = __ldg(a.ctab + 24 * (size_t)q + lane);
        }
        // the node order of corner lane of the site's cell (lane < 8), and this reflection's zone
        // points grouped by cell
        int my_ord = 0;
        if (lane < 8) {
            const int c = pcx + 2 * pcy + 4 * pcz, k = lane;
            const int lx = (c & 1) + (k & 1), ly = ((c >> 1) & 1) + ((k >> 1) & 1), lz = (c >> 2) + (k >> 2);
            const int rx = pcx ? lx : 2 - lx, ry = pcy ? ly : 2 - ly, rz = pcz ? lz : 2 - lz;
            my_ord = sch[rx + 3 * ry + 9 * rz];
        }
        const uint8_t *plist = plist_all + 32 * refl, *cend = cend_all + 8 * refl;
        {
            using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
            V *kv = reinterpret_cast<V *>(Kb);
            const V zero{};
            for (int i = lane; i < (int)(ZSLOT_CAP * ZBLK * sizeof(T) / 16); i += 32) kv[i] = zero;
        }
        __syncwarp();
        if (lane < 6) {
            const int o = lane < 3 ? 0 : lane < 5 ? ordB : ordC, r = lane < 3 ? lane : lane == 3 ? 1 : 2;
            Kb[sch[ZS_DIAG + o] * ZBLK + 5 * r] = T(1);   // (r, r) of the diagonal block
        }
        const int pa = x & 1, pb = y & 1, pcq = z & 1;

        // block Cholesky in the static order; a non-positive pivot (the smallest one is kept) or a
        // non-finite G marks the trial as failed
        T pmin = T(1);
        // the 3x3 diagonal factor of step k from reciprocal square roots (one special-function
        // operation per pivot instead of a square root and a division); every lane holds the
        // off-diagonal entries and the reciprocal pivots, which is all the column solves use
        T l10, l20, l21, i00, i11, i22;
        auto factor = [&](const T *Dk) {
            T r0[4], r1v[4], r2[4];
            ld4(Dk, r0);
            ld4(Dk + 4, r1v);
            ld4(Dk + 8, r2);
            const T a00 = r0[0];
            i00 = zrsqrt(a00);
            l10 = r1v[0] * i00;
            l20 = r2[0] * i00;
            const T a11 = r1v[1] - l10 * l10;
            i11 = zrsqrt(a11);
            l21 = (r2[1] - l20 * l10) * i11;
            const T a22 = r2[2] - l20 * l20 - l21 * l21;
            i22 = zrsqrt(a22);
            pmin = fmin(pmin, fmin(a00, fmin(a11, a22)));
        };
        // row r of a column block (I, k): L_Ik = C_Ik L_kk^-T
        auto solve_row = [&](T (&v)[4]) {
            const T x0 = v[0] * i00;
            const T x1 = (v[1] - x0 * l10) * i11;
            const T x2 = (v[2] - x0 * l20 - x1 * l21) * i22;
            v[0] = x0;
            v[1] = x1;
            v[2] = x2;
        };
        // C_IJ -= L_Ik L_Jk^T on the rows of C held in cv, stored back
        auto update = [&](T *C, const T (&li)[3][4], const T (&lj)[3][4], T (&cv)[3][4]) {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    cv[r][c] = fma(-li[r][0], lj[c][0], cv[r][c]);
                    cv[r][c] = fma(-li[r][1], lj[c][1], cv[r][c]);
                    cv[r][c] = fma(-li[r][2], lj[c][2], cv[r][c]);
                }
                st4(C + 4 * r, cv[r]);
            }
        };
        // One round of block updates, a warp barrier after it.  No column block or factor is
        // read after its own step (the border's Schur complement, not a stored factor, gives
        // G), so each update lane factors its step's pivot and forms the two column blocks it
        // needs from the unsolved ones (the same arithmetic as a column solve); nothing of the
        // column is stored.  The host schedules every update into the earliest round after
        // the updates it reads (its pivot's and its column blocks' last updates, its target's
        // previous one), so a round may hold the updates of several steps, and every block
        // gets its updates in step order, as in a step-by-step elimination.
        auto elim_round = [&](int r) {
            const uint2 it = *reinterpret_cast<const uint2 *>(sch + ZS_RND + 128 * r + 4 * lane);
            const uint32_t sC = it.x & 0xffffu;
            if (sC != 0xffffu) {
                factor(Kb + (it.y >> 16) * ZBLK);
                T *C = Kb + sC * ZBLK;
                const T *LI = Kb + (it.x >> 16) * ZBLK, *LJ = Kb + (it.y & 0xffffu) * ZBLK;
                T li[3][4], lj[3][4], cv[3][4];
#pragma unroll
                for (int rr = 0; rr < 3; ++rr) {
                    ld4(LI + 4 * rr, li[rr]);
                    ld4(LJ + 4 * rr, lj[rr]);
                    ld4(C + 4 * rr, cv[rr]);
                }
#pragma unroll
                for (int rr = 0; rr < 3; ++rr) {
                    solve_row(li[rr]);
                    solve_row(lj[rr]);
                }
                update(C, li, lj, cv);
            }
            __syncwarp();
        };

        // assembly: K = sum of B^T C' B over the zone's points (element tables per orientation and
        // position); the points of one zone cell share its DOF map, so they are summed in registers
        // and scattered once per cell.  The element rows are read from L2 three points ahead of
        // their sum (three register buffers in rotation), so that the loads overlap.
        {
            T acc[NJ], b0[NJ], b1[NJ], b2[NJ];
#pragma unroll
            for (int j = 0; j < NJ; ++j) acc[j] = T(0);
            // element rows are padded with zeros to 320 entries, so every lane loads NJ of them
            auto fetch = [&](int s, T(&v)[NJ]) {
                const uint32_t qs = __shfl_sync(FULL, asm_q, s), pos = __shfl_sync(FULL, my_pos, s);
                const T *ke = a.ktab + ((size_t)qs * 8 + pos) * ZROW + lane;
#pragma unroll
                for (int j = 0; j < NJ; ++j) v[j] = ldg_stream(ke + 32 * j);
            };
            fetch(plist[0], b0);
            fetch(plist[1], b1);
            fetch(plist[2], b2);
            int c = 0, cn = cend[0];
            // add point u (held in buf), scatter when it closes its zone cell, refill buf with point u + 3
            auto step = [&](int u, T(&buf)[NJ]) {
#pragma unroll
                for (int j = 0; j < NJ; ++j) acc[j] += buf[j];
                if (u + 3 < 27) fetch(plist[u + 3], buf);
                if (u + 1 == cn) {
                    // the entries' places in the block slots for this reflection and zone cell
                    // (zone_scatter_table): padding entries and those of fixed DOFs go to the
                    // unused last slot, so the scatter has no branches
                    const uint16_t *sc = a.scatter + (size_t)(refl * 8 + c) * ZROW + lane;
#pragma unroll
                    for (int j = 0; j < NJ; ++j) Kb[__ldg(sc + 32 * j)] += acc[j];
#pragma unroll
                    for (int j = 0; j < NJ; ++j) acc[j] = T(0);
                    __syncwarp();
                    // the cell's outer corner (reflected cell rc, node (2 rcx, 2 rcy, 2 rcz)) lies
                    // in this cell alone, so its blocks are complete: eliminate it now (steps
                    // 1..6; node A and the site cell's corner excepted) while the next cell's
                    // rows are in flight.  Later cells add to the blocks it updates.
                    const int rc = c ^ (~refl & 7);
                    const int kc = sch[2 * (rc & 1) + 6 * ((rc >> 1) & 1) + 18 * (rc >> 2)];
                    if (kc >= 1 && kc <= 6) elim_round(kc - 1);
                    ++c;
                    cn = c < 8 ? cend[c] : 27;
                }
            };
            for (int u = 0; u < 27; u += 3) {
                step(u, b0);
                step(u + 1, b1);
                step(u + 2, b2);
            }
        }
        __syncwarp();

        // the site's strain e0 = Ebar + B_p u from its cell's nodal displacements (lane =
        // 3 corner + alpha), dC in shared memory, w = dC e0, and the border: row 0 of block
        // (27, order of corner c) holds f = B_p^T w on that corner's DOFs (lane 3 c + alpha)
        T e0[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        if (lane < 24) {
            const int cr = lane / 3, al = lane % 3;
            T g[3];
            corner_grad<T>(pa, pb, pcq, cr & 1, (cr >> 1) & 1, cr >> 2, g);
#pragma unroll
            for (int k = 0; k < 6; ++k) e0[k] = bt_entry<T>(g, al, k) * uv;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) e0[k] += __shfl_xor_sync(FULL, e0[k], o);
        {
            T eb[6];
            load_ebar<T>(R.st, eb);
#pragma unroll
            for (int k = 0; k < 6; ++k) e0[k] = eb[k] + e0[k];
        }
        if (lane < 21) {
            int i = 0, rem = lane;
            while (rem >= 6 - i) {
                rem -= 6 - i;
                ++i;
            }
            const int j = i + rem;
            const T d = c_new - c_old;
            dCs[6 * i + j] = d;
            dCs[6 * j + i] = d;
        }
        __syncwarp();
        T wl = T(0);
        if (lane < 6) {
#pragma unroll
            for (int k = 0; k < 6; ++k) wl += dCs[6 * lane + k] * e0[k];
        }
        T w[6];
#pragma unroll
        for (int v = 0; v < 6; ++v) w[v] = __shfl_sync(FULL, wl, v);
        const int ordc = __shfl_sync(FULL, my_ord, (lane / 3) & 7);
        if (lane < 24) {
            const int cr = lane / 3, al = lane % 3;
            T g[3];
            corner_grad<T>(pa, pb, pcq, cr & 1, (cr >> 1) & 1, cr >> 2, g);
            T fv = T(0);
#pragma unroll
            for (int v = 0; v < 6; ++v) fv += bt_entry<T>(g, al, v) * w[v];
            Kb[sch[ZS_BIDX + ZN * 27 + ordc] * ZBLK + al] = fv;
        }
        __syncwarp();

        // the remaining steps (edges and face centres, the site cell) in their scheduled rounds;
        // the corners were eliminated during the assembly
        const int nround = sch[ZS_NROUND];
        for (int r = 6; r < nround; ++r) elim_round(r);
        __syncwarp();

        // -f . K'^+ f, left in the first entry of the pseudo-node's diagonal block; a pivot that
        // was not positive (the smallest is kept) or a result that overflowed or is not a
        // number fails the trial
        const T kf = Kb[sch[ZS_BIDX + ZN * 27 + 27] * ZBLK];
        const bool ok = __all_sync(FULL, pmin > T(0)) && fabs(kf) <= T(3.0e38);
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
        if (lane == 0) {
            T f = T(0);
#pragma unroll
            for (int i = 0; i < 6; ++i) f += e0[i] * w[i];
            f += kf;
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

namespace {

// One block update C_IJ -= L_Ik L_Jk^T of elimination step k, by block ids ZN * I + J.
struct ZUpdate {
    int C = -1, I = -1, J = -1, D = -1;   // target, column blocks (I, k) and (J, k), pivot (k, k)
};

// Shared-memory layout of the factorisation.  A block's row r of slot s is the 16-byte
// unit 3 s + r of the warp's block area, so the eight lanes of a quarter warp that load
// row r of distinct blocks s hit distinct bank groups exactly when their s are distinct
// mod 8 (3 is odd); lanes loading the same block share the access.  The cost of a layout
// is the number of shared-memory wavefronts of the block loads and stores of the
// updates (32 lanes, four quarters per 16-byte access), with the slots of the blocks and
// the lane of each update within its round as the free choices; neither changes any
// arithmetic (each block gets its updates in the same order, and where it is stored does
// not matter), so every layout gives the same bits.
struct ZoneLayout {
    std::vector<std::vector<ZUpdate>> rounds;   // per round 32 lanes (C < 0: no update)
    std::vector<int> slot_of;                   // ZN * I + J -> slot (-1 if structurally zero)
};

int quarter_wavefronts(const int *s, int n) {
    // distinct slots per residue mod 8 among the quarter's lanes; the largest count
    int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0}, w = 0;
    for (int i = 0; i < n; ++i) {
        bool seen = false;
        for (int j = 0; j < i; ++j) seen = seen || s[j] == s[i];
        if (!seen) w = std::max(w, ++cnt[s[i] & 7]);
    }
    return w;
}

long round_cost(const ZoneLayout &L, int r) {
    long c = 0;
    int s[8];
    const auto &u = L.rounds[r];
    for (int q = 0; q < 32; q += 8)
        for (int which = 0; which < 4; ++which) {
            int n = 0;
            for (int i = q; i < q + 8; ++i) {
                const ZUpdate &x = u[i];
                if (x.C < 0) continue;
                s[n++] = L.slot_of[which == 0 ? x.C : which == 1 ? x.I : which == 2 ? x.J : x.D];
            }
            if (n) c += quarter_wavefronts(s, n) * (which == 0 ? 6 : 3);   // C: 3 loads + 3 stores
        }
    return c;
}

// Simulated annealing over slot swaps and swaps of two lanes of one round (fixed seed,
// splitmix64; a few tenths of a second, once per process).
void optimise_layout(ZoneLayout &L, int nslots) {
    uint64_t st = 0x5EEDC0DE12345ull;
    auto rnd = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    const int nr = (int)L.rounds.size();
    std::vector<std::vector<int>> rounds_of(nslots);   // rounds whose cost involves a slot
    for (int r = 0; r < nr; ++r) {
        std::vector<int> ss;
        for (const ZUpdate &x : L.rounds[r])
            if (x.C >= 0)
                for (int b : {x.C, x.I, x.J, x.D}) ss.push_back(L.slot_of[b]);
        std::sort(ss.begin(), ss.end());
        ss.erase(std::unique(ss.begin(), ss.end()), ss.end());
        for (int x : ss) rounds_of[x].push_back(r);
    }
    std::vector<int> owner(nslots, -1);   // slot -> ZN I + J
    for (int b = 0; b < ZN * ZN; ++b)
        if (L.slot_of[b] >= 0) owner[L.slot_of[b]] = b;
    std::vector<long> cost(nr);
    for (int r = 0; r < nr; ++r) cost[r] = round_cost(L, r);
    double T = 2.0;
    for (int it = 0; it < 120000; ++it) {
        if (rnd() & 1) {
            const int a = (int)(rnd() % nslots), b = (int)(rnd() % nslots);
            if (a == b || owner[a] < 0 || owner[b] < 0) continue;
            std::vector<int> rs = rounds_of[a];
            rs.insert(rs.end(), rounds_of[b].begin(), rounds_of[b].end());
            std::sort(rs.begin(), rs.end());
            rs.erase(std::unique(rs.begin(), rs.end()), rs.end());
            long before = 0, after = 0;
            for (int r : rs) before += cost[r];
            std::swap(L.slot_of[owner[a]], L.slot_of[owner[b]]);
            std::vector<long> nc(rs.size());
            for (size_t i = 0; i < rs.size(); ++i) after += (nc[i] = round_cost(L, rs[i]));
            if (after <= before || (double)(rnd() >> 11) * 0x1.0p-53 < std::exp((before - after) / T)) {
                std::swap(owner[a], owner[b]);
                std::swap(rounds_of[a], rounds_of[b]);
                for (size_t i = 0; i < rs.size(); ++i) cost[rs[i]] = nc[i];
            } else {
                std::swap(L.slot_of[owner[a]], L.slot_of[owner[b]]);
            }
        } else {
            const int r = (int)(rnd() % nr);
            const int a = (int)(rnd() % 32), b = (int)(rnd() % 32);
            if (a == b || (L.rounds[r][a].C < 0 && L.rounds[r][b].C < 0)) continue;
            std::swap(L.rounds[r][a], L.rounds[r][b]);
            const long nc = round_cost(L, r);
            if (nc <= cost[r] || (double)(rnd() >> 11) * 0x1.0p-53 < std::exp((cost[r] - nc) / T))
                cost[r] = nc;
            else
                std::swap(L.rounds[r][a], L.rounds[r][b]);
        }
        T = std::max(0.05, T * 0.99995);
    }
}

}  // namespace

// Elimination schedule of the zone's 27 nodes in the reflected frame (the
// site's cell = nodes with all coordinates in {1,2}); layout at the top of this
// file.  Nodes share a block of K when they lie in a common zone cell
// (Chebyshev distance <= 1); the symbolic factorisation adds the fill of each
// step.  The outer corners' steps (1..6) are one round each, run during the
// assembly; the updates of the later steps are list-scheduled into rounds of 32
// lanes, each as early as the updates it reads allow (longest remaining chain
// first).  Every block of the filled lower triangle gets a storage slot, placed
// (with the lane of each update) by optimise_layout to spread the lanes' block
// accesses over the shared-memory banks.  Built once per process.
std::vector<uint16_t> zone_schedule_build();

std::vector<uint16_t> zone_schedule() {
    static std::once_flag once;
    static std::vector<uint16_t> table;
    std::call_once(once, [] { table = zone_schedule_build(); });
    return table;
}

std::vector<uint16_t> zone_schedule_build() {
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
    // the nine edge nodes and three face centres outside the site's cell, in the order with
    // the fewest block updates (found by exhaustive local search over the orders of these 12
    // nodes): 576 block updates, against 696 with all edges before the face centres.  Node
    // B = (1,0,0) (y, z fixed) and node C = (0,1,0) (z fixed) are among them; any order of a
    // positive definite matrix gives positive pivots.
    for (int n : {7, 1, 21, 4, 3, 5, 15, 9, 12, 19, 11, 10}) order.push_back(n);
    for (int n = 0; n < 27; ++n)
        if (cls(n) == 3) order.push_back(n);
    // the real nodes share a block when they lie in a common zone cell (Chebyshev distance
    // <= 1); the border pseudo-node (order 27) shares one with the site cell's nodes (orders
    // 19..26).  Node A (order 0) has all its DOFs held fixed: its
    // row and column of K are zero but for the unit diagonal, so it shares no block and its
    // elimination step is empty (the kernel starts at step 1).
    bool pat[ZN][ZN];
    for (int i = 0; i < ZN; ++i)
        for (int j = 0; j < ZN; ++j) {
            if (i >= 27 || j >= 27) {
                pat[i][j] = std::min(i, j) >= 19;
                continue;
            }
            if ((i == 0) != (j == 0)) {
                pat[i][j] = false;
                continue;
            }
            int dmax = 0;
            for (int d = 0; d < 3; ++d) dmax = std::max(dmax, std::abs(co(order[i], d) - co(order[j], d)));
            pat[i][j] = dmax <= 1;
        }
    // symbolic elimination of the 27 real nodes (the pseudo-node is never eliminated)
    std::vector<std::vector<ZUpdate>> up(27);
    for (int k = 0; k < 27; ++k) {
        std::vector<int> nb;
        for (int i = k + 1; i < ZN; ++i)
            if (pat[i][k]) nb.push_back(i);
        for (int I : nb)
            for (int J : nb)
                if (J <= I) {
                    up[k].push_back({ZN * I + J, ZN * I + k, ZN * J + k, (ZN + 1) * k});
                    pat[I][J] = pat[J][I] = true;
                }
    }
    ZoneLayout L;
    // steps 1..6 (the outer corners): one round each
    for (int k = 1; k <= 6; ++k) {
        if (up[k].size() > 32) return {};
        std::vector<ZUpdate> r(32);
        for (size_t i = 0; i < up[k].size(); ++i) r[i] = up[k][i];
        L.rounds.push_back(r);
    }
    // steps 7..26: an update reads its pivot and its two column blocks after their last
    // updates and its target after the target's previous update
    std::vector<ZUpdate> items;
    std::vector<int> step_of;
    for (int k = 7; k < 27; ++k)
        for (const ZUpdate &x : up[k]) {
            items.push_back(x);
            step_of.push_back(k);
        }
    const int ni = (int)items.size();
    std::vector<std::vector<int>> deps(ni), succ(ni);
    {
        std::vector<int> last(ZN * ZN, -1);   // block -> latest update of it among the items so far
        for (int i = 0; i < ni; ++i) {
            for (int b : {items[i].D, items[i].I, items[i].J, items[i].C})
                if (last[b] >= 0) deps[i].push_back(last[b]);
            last[items[i].C] = i;
        }
        for (int i = 0; i < ni; ++i)
            for (int d : deps[i]) succ[d].push_back(i);
    }
    // Items are in step order and an update's target is updated only by earlier steps, so
    // "latest so far" is the last update before this step for the pivot, the column blocks
    // and the target alike.  Chain lengths to the end, then greedy rounds.
    std::vector<int> chain(ni, 1);
    for (int i = ni - 1; i >= 0; --i)
        for (int s2 : succ[i]) chain[i] = std::max(chain[i], chain[s2] + 1);
    std::vector<int> round_of(ni, -1);
    int left = ni;
    for (int r = 0; left > 0; ++r) {
        std::vector<int> ready;
        for (int i = 0; i < ni; ++i) {
            if (round_of[i] >= 0) continue;
            bool ok = true;
            for (int d : deps[i]) ok = ok && round_of[d] >= 0 && round_of[d] < r;
            if (ok) ready.push_back(i);
        }
        std::stable_sort(ready.begin(), ready.end(), [&](int x, int y) { return chain[x] > chain[y]; });
        if (ready.size() > 32) ready.resize(32);
        std::vector<ZUpdate> rr(32);
        for (size_t l = 0; l < ready.size(); ++l) {
            rr[l] = items[ready[l]];
            round_of[ready[l]] = r;
        }
        left -= (int)ready.size();
        L.rounds.push_back(rr);
        if (r > 4 * ni) return {};
    }
    L.slot_of.assign(ZN * ZN, -1);
    int slots = 0;
    for (int I = 0; I < ZN; ++I)
        for (int J = 0; J <= I; ++J)
            if (pat[I][J]) L.slot_of[ZN * I + J] = slots++;
    if (slots > ZSLOT_CAP - 1) return {};   // the last slot stays free (ZTRASH)
    optimise_layout(L, slots);
    const size_t nround = L.rounds.size();
    if (ZS_RND + 128 * nround > (size_t)ZSCHED_CAP) return {};
    std::vector<uint16_t> t(ZS_RND + 128 * nround, 0);
    for (int i = 0; i < 27; ++i) t[order[i]] = (uint16_t)i;
    t[ZS_NROUND] = (uint16_t)nround;
    for (int I = 0; I < ZN; ++I)
        for (int J = 0; J < ZN; ++J)
            t[ZS_BIDX + ZN * I + J] = L.slot_of[ZN * I + J] >= 0 ? (uint16_t)L.slot_of[ZN * I + J] : (uint16_t)0xffff;
    for (int k = 0; k < 27; ++k) t[ZS_DIAG + k] = t[ZS_BIDX + (ZN + 1) * k];
    for (size_t r = 0; r < nround; ++r)
        for (int l = 0; l < 32; ++l) {
            const ZUpdate &x = L.rounds[r][l];
            uint16_t *e = &t[ZS_RND + 128 * r + 4 * l];
            if (x.C < 0) {
                e[0] = e[1] = e[2] = e[3] = 0xffff;
                continue;
            }
            e[0] = (uint16_t)L.slot_of[x.C];
            e[1] = (uint16_t)L.slot_of[x.I];
            e[2] = (uint16_t)L.slot_of[x.J];
            e[3] = (uint16_t)L.slot_of[x.D];
        }
    return t;
}

// Where each entry of a zone cell's summed element matrix goes in the block slots:
// for reflection rf = pcx + 2 pcy + 4 pcz (the site's zone cell), zone cell c and
// upper-triangle entry t of the 24 x 24 element matrix (element DOF 3 corner + alpha),
// the float offset slot(o1, o2) * 12 + 4 a1 + a2 of its lower-triangle place, or the
// unused last slot when either DOF is one of the six held fixed.  Rows padded to 320
// entries, the padding pointing at the unused slot as well.
std::vector<uint16_t> zone_scatter_table(const std::vector<uint16_t> &t) {
    std::vector<uint16_t> out((size_t)64 * ZROW, (uint16_t)ZTRASH);
    const int ordB = t[1], ordC = t[3];
    for (int rf = 0; rf < 8; ++rf) {
        const int pcx = rf & 1, pcy = (rf >> 1) & 1, pcz = rf >> 2;
        for (int c = 0; c < 8; ++c) {
            auto order_of = [&](int k) {
                const int lx = (c & 1) + (k & 1), ly = ((c >> 1) & 1) + ((k >> 1) & 1), lz = (c >> 2) + (k >> 2);
                const int rx = pcx ? lx : 2 - lx, ry = pcy ? ly : 2 - ly, rz = pcz ? lz : 2 - lz;
                return (int)t[rx + 3 * ry + 9 * rz];
            };
            int e = 0;
            for (int e1 = 0; e1 < 24; ++e1)
                for (int e2 = e1; e2 < 24; ++e2, ++e) {
                    int o1 = order_of(e1 / 3), a1 = e1 % 3, o2 = order_of(e2 / 3), a2 = e2 % 3;
                    const bool f1 = o1 == 0 || (o1 == ordB && a1 >= 1) || (o1 == ordC && a1 == 2);
                    const bool f2 = o2 == 0 || (o2 == ordB && a2 >= 1) || (o2 == ordC && a2 == 2);
                    if (f1 || f2) continue;
                    if (o1 < o2 || (o1 == o2 && a1 < a2)) {
                        std::swap(o1, o2);
                        std::swap(a1, a2);
                    }
                    out[(size_t)(rf * 8 + c) * ZROW + e] = (uint16_t)(t[ZS_BIDX + ZN * o1 + o2] * ZBLK + 4 * a1 + a2);
                }
        }
    }
    return out;
}

// Element stiffness V B^T C'(q) B (V = 1 voxel) of a point at local position
// pos = a + 2b + 4c of its cell, in element DOF order 3 corner + alpha, upper
// triangle row-major (300 values, padded with zeros to ZROW), for every orientation.
void zone_element_tables(const double *Cv, int Q, std::vector<double> &out) {
    out.assign((size_t)Q * 8 * ZROW, 0.0);
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
            double *o = &out[((size_t)q * 8 + pos) * ZROW];
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
