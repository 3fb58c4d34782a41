/*
 * hmc_oracle.c -- plain, slow, FP64 CPU oracle of the hybrid Monte Carlo (HMC)
 * hot path of Zhang, Bartel & Lusk, "Parallelized Hybrid Monte Carlo Simulation
 * of Stress-Induced Texture Evolution".
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA library; the two
 * are compared element by element on the same seeded inputs.
 *
 * Every loop is written in the order the paper states the method, with no
 * blocking, fusion or reordering.  All floating point is double.
 *
 * Layouts (all natural, x fastest):
 *   site   (x,y,z)  -> x + nx*(y + ny*z)                  voxel = MC site = material point
 *   node   (i,j,k)  -> i + nbx*(j + nby*k), nb* = n* / 2     background mesh node at voxel corner (2i,2j,2k)
 *   tensors in Voigt order (11,22,33,23,13,12); strain with engineering shear.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11: ten rounds of two 32x32->64 multiplies, with the */
/* Weyl key schedule between rounds.  The Monte Carlo trial draw (the paper's */
/* random site trial, Sec. "Hybrid Monte Carlo Methodology") is keyed by     */
/* (seed) and counted by (site, sweep, replica).                              */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* Orientation tables (Sec. "Elastic Deformation", Eqs. 16-18).              */
/* ------------------------------------------------------------------------- */

static void mat3_mul(const double a[9], const double b[9], double c[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += a[3 * i + k] * b[3 * k + j];
            c[3 * i + j] = s;
        }
}

/* A = B C D with B = Rz(phi), C = Ry(theta), D = Rz(psi) (Eq. 18, z-y-z Euler
 * angles).  A is row-major; its columns are the crystal axes written in the
 * sample frame, so a crystal-frame vector v maps to A v. */
void orc_euler_zyz_to_A(double phi, double theta, double psi, double A[9])
{
    double cf = cos(phi), sf = sin(phi), ct = cos(theta), st = sin(theta);
    double cp = cos(psi), sp = sin(psi);
    double B[9] = {cf, -sf, 0.0, sf, cf, 0.0, 0.0, 0.0, 1.0};
    double C[9] = {ct, 0.0, st, 0.0, 1.0, 0.0, -st, 0.0, ct};
    double D[9] = {cp, -sp, 0.0, sp, cp, 0.0, 0.0, 0.0, 1.0};
    double BC[9];
    mat3_mul(B, C, BC);
    mat3_mul(BC, D, A);
}

/* Crystal-frame cubic stiffness tensor component C_mnop from the three
 * independent constants (Sec. "Elastic Deformation": cubic symmetry). */
static double cubic_tensor(double c11, double c12, double c44, int m, int n, int o, int p)
{
    if (m == n && o == p) return (m == o) ? c11 : c12;
    if (m != n && ((m == o && n == p) || (m == p && n == o))) return c44;
    return 0.0;
}

static const int VOIGT_I[6] = {0, 1, 2, 1, 0, 0};
static const int VOIGT_J[6] = {0, 1, 2, 2, 2, 1};

/* Rotated stiffness, Eq. 17 read as C'_ijkl = sum_mnop A_im A_jn A_ko A_lp C_mnop
 * (the printed right-hand side repeats the free indices), written out as the
 * literal 81-term sum for each of the 81 components, then stored as the
 * 6x6 Voigt matrix (engineering shear strain): C[6*I+J]. */
void orc_rotated_stiffness(double c11, double c12, double c44, const double A[9], double Cv[36])
{
    double Ct[81];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    double s = 0.0;
                    for (int m = 0; m < 3; ++m)
                        for (int n = 0; n < 3; ++n)
                            for (int o = 0; o < 3; ++o)
                                for (int p = 0; p < 3; ++p)
                                    s += A[3 * i + m] * A[3 * j + n] * A[3 * k + o] * A[3 * l + p] *
                                         cubic_tensor(c11, c12, c44, m, n, o, p);
                    Ct[27 * i + 9 * j + 3 * k + l] = s;
                }
    for (int I = 0; I < 6; ++I)
        for (int J = 0; J < 6; ++J)
            Cv[6 * I + J] = Ct[27 * VOIGT_I[I] + 9 * VOIGT_J[I] + 3 * VOIGT_I[J] + VOIGT_J[J]];
}

/* Compliance S = C^-1 of a 6x6 Voigt stiffness (engineering shear), by
 * Gauss-Jordan elimination with partial pivoting.  Returns 0 on success,
 * -1 if C is singular. */
int orc_invert6(const double Cv[36], double Sv[36])
{
    double a[6][12];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 12; ++j) a[i][j] = (j < 6) ? Cv[6 * i + j] : (j - 6 == i ? 1.0 : 0.0);
    for (int col = 0; col < 6; ++col) {
        int piv = col;
        for (int r = col + 1; r < 6; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0) return -1;
        if (piv != col)
            for (int j = 0; j < 12; ++j) {
                double t = a[col][j];
                a[col][j] = a[piv][j];
                a[piv][j] = t;
            }
        double d = a[col][col];
        for (int j = 0; j < 12; ++j) a[col][j] /= d;
        for (int r = 0; r < 6; ++r) {
            if (r == col) continue;
            double f = a[r][col];
            if (f == 0.0) continue;
            for (int j = 0; j < 12; ++j) a[r][j] -= f * a[col][j];
        }
    }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) Sv[6 * i + j] = a[i][j + 6];
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Time-explicit material point method (Sec. "Elastic Deformation").         */
/* Material points are the voxel centres; the background mesh has cells of   */
/* two voxels per edge, i.e. two material points per cell in each direction   */
/* (the particle layout of the Appendix), periodic.  Trilinear shape          */
/* functions; the strain of a point is the mean strain Ebar plus the          */
/* symmetric gradient of the periodic nodal displacement field.               */
/* ------------------------------------------------------------------------- */

static const double MPM_H = 2.0;   /* cell edge in voxels            */
static const double MPM_VP = 1.0;  /* particle volume (one voxel)    */
static const double MPM_RHO = 1.0; /* density (quasi-static, scaled) */

static inline int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }

static inline int64_t node_index(int i, int j, int k, int nbx, int nby, int nbz)
{
    return (int64_t)wrap(i, nbx) + (int64_t)nbx * ((int64_t)wrap(j, nby) + (int64_t)nby * wrap(k, nbz));
}

/* Shape function N_I and its gradient for the I-th corner (I = di + 2 dj + 4 dk)
 * of the cell holding the point at local coordinates xi in [0,1]^3. */
static void trilinear(int di, int dj, int dk, const double xi[3], double *N, double gradN[3])
{
    double n0 = di ? xi[0] : 1.0 - xi[0];
    double n1 = dj ? xi[1] : 1.0 - xi[1];
    double n2 = dk ? xi[2] : 1.0 - xi[2];
    double d0 = (di ? 1.0 : -1.0) / MPM_H;
    double d1 = (dj ? 1.0 : -1.0) / MPM_H;
    double d2 = (dk ? 1.0 : -1.0) / MPM_H;
    *N = n0 * n1 * n2;
    gradN[0] = d0 * n1 * n2;
    gradN[1] = n0 * d1 * n2;
    gradN[2] = n0 * n1 * d2;
}

static void point_cell(int x, int y, int z, int *cx, int *cy, int *cz, double xi[3])
{
    *cx = x / 2; *cy = y / 2; *cz = z / 2;
    xi[0] = ((x & 1) + 0.5) / MPM_H;
    xi[1] = ((y & 1) + 0.5) / MPM_H;
    xi[2] = ((z & 1) + 0.5) / MPM_H;
}

/* Strain of material point (x,y,z): eps = Ebar + sym(sum_I u_I (x) gradN_I). */
void orc_point_strain(int nx, int ny, int nz, const double *u, const double Ebar[6],
                      int x, int y, int z, double eps[6])
{
    int nbx = nx / 2, nby = ny / 2, nbz = nz / 2, cx, cy, cz;
    double xi[3], G[3][3] = {{0}};
    point_cell(x, y, z, &cx, &cy, &cz, xi);
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                double N, g[3];
                trilinear(di, dj, dk, xi, &N, g);
                int64_t I = node_index(cx + di, cy + dj, cz + dk, nbx, nby, nbz);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) G[a][b] += u[3 * I + a] * g[b];
            }
    eps[0] = Ebar[0] + G[0][0];
    eps[1] = Ebar[1] + G[1][1];
    eps[2] = Ebar[2] + G[2][2];
    eps[3] = Ebar[3] + G[1][2] + G[2][1];
    eps[4] = Ebar[4] + G[0][2] + G[2][0];
    eps[5] = Ebar[5] + G[0][1] + G[1][0];
}

/* Strain of every point (N x 6). */
void orc_strain_field(int nx, int ny, int nz, const double *u, const double Ebar[6], double *eps)
{
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t p = (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
                orc_point_strain(nx, ny, nz, u, Ebar, x, y, z, eps + 6 * p);
            }
}

/* Hooke's law, Eq. 1: S = C eps with the point's rotated stiffness. */
static void hooke(const double *C, const double eps[6], double sig[6])
{
    for (int I = 0; I < 6; ++I) {
        double s = 0.0;
        for (int J = 0; J < 6; ++J) s += C[6 * I + J] * eps[J];
        sig[I] = s;
    }
}

void orc_point_stress(int nx, int ny, int nz, const uint16_t *spin, const double *Ctab,
                      const double *u, const double Ebar[6], int x, int y, int z, double sig[6])
{
    double eps[6];
    orc_point_strain(nx, ny, nz, u, Ebar, x, y, z, eps);
    int64_t p = (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
    hooke(Ctab + 36 * (int64_t)spin[p], eps, sig);
}

/* Internal nodal force f_I = - sum_p V_p sigma_p . gradN_I(x_p): strain and
 * stress at every material point, mapped back to the nodes. */
void orc_internal_force(int nx, int ny, int nz, const uint16_t *spin, const double *Ctab,
                        const double *u, const double Ebar[6], double *f)
{
    int nbx = nx / 2, nby = ny / 2, nbz = nz / 2;
    int64_t nn = (int64_t)nbx * nby * nbz;
    memset(f, 0, sizeof(double) * 3 * nn);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double sig[6], xi[3];
                int cx, cy, cz;
                orc_point_stress(nx, ny, nz, spin, Ctab, u, Ebar, x, y, z, sig);
                double S[3][3] = {{sig[0], sig[5], sig[4]}, {sig[5], sig[1], sig[3]}, {sig[4], sig[3], sig[2]}};
                point_cell(x, y, z, &cx, &cy, &cz, xi);
                for (int dk = 0; dk < 2; ++dk)
                    for (int dj = 0; dj < 2; ++dj)
                        for (int di = 0; di < 2; ++di) {
                            double N, g[3];
                            trilinear(di, dj, dk, xi, &N, g);
                            int64_t I = node_index(cx + di, cy + dj, cz + dk, nbx, nby, nbz);
                            for (int a = 0; a < 3; ++a) {
                                double s = 0.0;
                                for (int b = 0; b < 3; ++b) s += S[a][b] * g[b];
                                f[3 * I + a] -= MPM_VP * s;
                            }
                        }
            }
}

/* Internal force of one node (i,j,k): the same sum as orc_internal_force,
 * gathered over the 64 points of the node's eight cells. */
void orc_node_force(int nx, int ny, int nz, const uint16_t *spin, const double *Ctab, const double *u,
                    const double Ebar[6], int i, int j, int k, double f[3])
{
    f[0] = f[1] = f[2] = 0.0;
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                /* the cell that has this node as corner (di,dj,dk) */
                int cx = wrap(i - di, nx / 2), cy = wrap(j - dj, ny / 2), cz = wrap(k - dk, nz / 2);
                for (int lz = 0; lz < 2; ++lz)
                    for (int ly = 0; ly < 2; ++ly)
                        for (int lx = 0; lx < 2; ++lx) {
                            int x = 2 * cx + lx, y = 2 * cy + ly, z = 2 * cz + lz;
                            double sig[6], xi[3], N, g[3];
                            int ccx, ccy, ccz;
                            orc_point_stress(nx, ny, nz, spin, Ctab, u, Ebar, x, y, z, sig);
                            point_cell(x, y, z, &ccx, &ccy, &ccz, xi);
                            trilinear(di, dj, dk, xi, &N, g);
                            double S[3][3] = {{sig[0], sig[5], sig[4]}, {sig[5], sig[1], sig[3]}, {sig[4], sig[3], sig[2]}};
                            for (int a = 0; a < 3; ++a) {
                                double t = 0.0;
                                for (int b = 0; b < 3; ++b) t += S[a][b] * g[b];
                                f[a] -= MPM_VP * t;
                            }
                        }
            }
}

/* Lumped nodal mass m_I = sum_p rho V_p N_I(x_p). */
void orc_lumped_mass(int nx, int ny, int nz, double *m)
{
    int nbx = nx / 2, nby = ny / 2, nbz = nz / 2;
    int64_t nn = (int64_t)nbx * nby * nbz;
    memset(m, 0, sizeof(double) * nn);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double xi[3];
                int cx, cy, cz;
                point_cell(x, y, z, &cx, &cy, &cz, xi);
                for (int dk = 0; dk < 2; ++dk)
                    for (int dj = 0; dj < 2; ++dj)
                        for (int di = 0; di < 2; ++di) {
                            double N, g[3];
                            trilinear(di, dj, dk, xi, &N, g);
                            m[node_index(cx + di, cy + dj, cz + dk, nbx, nby, nbz)] += MPM_RHO * MPM_VP * N;
                        }
            }
}

/* One explicit step towards the quasi-static state: internal force from the
 * current displacement, damped velocity update, displacement update
 * (v <- (1 - damping) v + dt f / m;  u <- u + dt v).  f and m are caller
 * workspace of 3*nnodes and nnodes doubles. */
void orc_mpm_step(int nx, int ny, int nz, const uint16_t *spin, const double *Ctab, const double Ebar[6],
                  double *u, double *v, double dt, double damping, double *f, double *m)
{
    int64_t nn = (int64_t)(nx / 2) * (ny / 2) * (nz / 2);
    orc_internal_force(nx, ny, nz, spin, Ctab, u, Ebar, f);
    orc_lumped_mass(nx, ny, nz, m);
    for (int64_t I = 0; I < nn; ++I)
        for (int a = 0; a < 3; ++a) {
            v[3 * I + a] = (1.0 - damping) * v[3 * I + a] + dt * f[3 * I + a] / m[I];
            u[3 * I + a] = u[3 * I + a] + dt * v[3 * I + a];
        }
}

/* Stress at every point (N x 6) with the mean stress and the elastic energy
 * sum_p 1/2 V_p sigma_p . eps_p (Eq. 1). */
void orc_stress_field(int nx, int ny, int nz, const uint16_t *spin, const double *Ctab,
                      const double *u, const double Ebar[6], double *sig, double mean[6], double *energy)
{
    int64_t N = (int64_t)nx * ny * nz;
    double acc[6] = {0}, W = 0.0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t p = (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
                double eps[6], s[6];
                orc_point_strain(nx, ny, nz, u, Ebar, x, y, z, eps);
                hooke(Ctab + 36 * (int64_t)spin[p], eps, s);
                for (int c = 0; c < 6; ++c) {
                    sig[6 * p + c] = s[c];
                    acc[c] += s[c];
                    W += 0.5 * MPM_VP * s[c] * eps[c];
                }
            }
    for (int c = 0; c < 6; ++c) mean[c] = acc[c] / (double)N;
    *energy = W;
}

/* ------------------------------------------------------------------------- */
/* Potts Monte Carlo with the point-zone elastic shift.                      */
/* ------------------------------------------------------------------------- */

/* Elastic shift of the single-point constant-traction zone (Eqs. 6-8, read as
 * the change of potential energy of a dead-loaded point whose compliance goes
 * from S_old to S_new at fixed stress): w(S_old) - w(S_new), w = 1/2 s.S.s. */
double orc_point_zone_shift(const double *S_old, const double *S_new, const double sig[6])
{
    double w_old = 0.0, w_new = 0.0;
    for (int I = 0; I < 6; ++I)
        for (int J = 0; J < 6; ++J) {
            w_old += 0.5 * sig[I] * S_old[6 * I + J] * sig[J];
            w_new += 0.5 * sig[I] * S_new[6 * I + J] * sig[J];
        }
    return w_old - w_new;
}

/* Elastic shift of the single-point constant-strain zone (Eq. 8 read with the
 * point's strain held fixed, e = S_old s): the change of its energy density,
 * 1/2 e.(C_new - C_old).e. */
double orc_point_strain_shift(const double *S_old, const double *C_old, const double *C_new, const double sig[6])
{
    double e[6];
    for (int I = 0; I < 6; ++I) {
        e[I] = 0.0;
        for (int J = 0; J < 6; ++J) e[I] += S_old[6 * I + J] * sig[J];
    }
    double d = 0.0;
    for (int I = 0; I < 6; ++I)
        for (int J = 0; J < 6; ++J) d += 0.5 * e[I] * (C_new[6 * I + J] - C_old[6 * I + J]) * e[J];
    return d;
}

enum { ORC_ELASTIC_OFF = 0, ORC_ELASTIC_TRACTION = 1, ORC_ELASTIC_STRAIN = 3 };

/* Integer acceptance threshold of the Metropolis rule (Eq. 5) for an integer
 * bond-energy change k > 0: accept iff r1 < T(k), equivalent to
 * (r1 + 1/2) 2^-32 < exp(-k J / kT) for every 32-bit r1. */
double orc_accept_threshold(int k, double J, double kT)
{
    if (k <= 0) return 4294967296.0;
    if (!(kT > 0.0)) return 0.0;
    return ceil(exp(-(double)k * J / kT) * 4294967296.0 - 0.5);
}

enum { ORC_TRIAL_NEIGHBOR = 0, ORC_TRIAL_UNIFORM_Q = 1 };

/* One Monte Carlo trial at site (x,y,z) for sweep index mcs, against the
 * current spin field (Eqs. 4-5 with the elastic shift of Eqs. 8 and 13).
 * Returns 1 if the spin changes.  *q_new receives the trial state, *dH the
 * total change in MC energy units, *thresh the Metropolis threshold
 * -kT ln u (or -1 when the integer table decided).  sig_p is the site's
 * stress (6 values; unused when the elastic term is off). */
/* The two draws of the trial at site (x, y, z) of Monte Carlo step mcs: out[0]
 * picks the trial state, out[1] decides.  The four sites of one colour in the
 * same 2x2x2 block (origin x, y, z all even) share one Philox4x32-10 block:
 * counter (index of the block origin, mcs, replica, 2 + colour), key (seed lo,
 * seed hi); the site whose local corner index lx + 2 ly + 4 lz is the j-th
 * smallest among its colour's four takes word j.  Neighbour trials: out[0] is that
 * word w and out[1] the low 32 bits of 6 w (the neighbour index is the high
 * bits).  Trials over all orientations: out[1] is word j of a second block with
 * counter word 3 = 4 + colour. */
void orc_site_draws(int nx, int ny, int x, int y, int z, uint64_t seed, uint32_t mcs, uint32_t replica,
                    int trial_mode, uint32_t out[2])
{
    const int colour = (x + y + z) & 1;
    const int L = (x & 1) + 2 * (y & 1) + 4 * (z & 1);
    int j = 0;   /* corners of the same colour with a smaller local index */
    for (int m = 0; m < L; ++m)
        if ((((m & 1) + ((m >> 1) & 1) + (m >> 2)) & 1) == colour) ++j;
    const int64_t origin = (int64_t)(x & ~1) + (int64_t)nx * ((int64_t)(y & ~1) + (int64_t)ny * (z & ~1));
    uint32_t ctr[4] = {(uint32_t)origin, mcs, replica, 2u + (uint32_t)colour};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    out[0] = r[j];
    if (trial_mode == ORC_TRIAL_NEIGHBOR) {
        out[1] = (uint32_t)((uint64_t)r[j] * 6u);   /* mod 2^32 */
    } else {
        ctr[3] = 4u + (uint32_t)colour;
        orc_philox4x32_10(ctr, key, r);
        out[1] = r[j];
    }
}

int orc_site_trial_at(int nx, int ny, int nz, const uint16_t *spin, int x, int y, int z,
                      uint64_t seed, uint32_t mcs, uint32_t replica, double J, double kT,
                      int trial_mode, int Q, int elastic, double lambda, const double *Stab,
                      const double *Ctab, const double *sig_p, uint16_t *q_new, double *dH, double *thresh)
{
    int64_t p = (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
    uint32_t r[2];
    orc_site_draws(nx, ny, x, y, z, seed, mcs, replica, trial_mode, r);

    /* neighbours in the order -x, +x, -y, +y, -z, +z (periodic lattice) */
    uint16_t nb[6];
    nb[0] = spin[wrap(x - 1, nx) + (int64_t)nx * (y + (int64_t)ny * z)];
    nb[1] = spin[wrap(x + 1, nx) + (int64_t)nx * (y + (int64_t)ny * z)];
    nb[2] = spin[x + (int64_t)nx * (wrap(y - 1, ny) + (int64_t)ny * z)];
    nb[3] = spin[x + (int64_t)nx * (wrap(y + 1, ny) + (int64_t)ny * z)];
    nb[4] = spin[x + (int64_t)nx * (y + (int64_t)ny * wrap(z - 1, nz))];
    nb[5] = spin[x + (int64_t)nx * (y + (int64_t)ny * wrap(z + 1, nz))];

    uint16_t q = spin[p], qt;
    if (trial_mode == ORC_TRIAL_NEIGHBOR)
        qt = nb[(int)(((uint64_t)r[0] * 6u) >> 32)];
    else
        qt = (uint16_t)(((uint64_t)r[0] * (uint64_t)Q) >> 32);
    *q_new = qt;
    *thresh = -1.0;
    if (qt == q) {
        *dH = 0.0;
        return 0;
    }
    /* bond energy J * (number of unlike neighbours): change = J (n(q) - n(q')) */
    int n_old = 0, n_new = 0;
    for (int k = 0; k < 6; ++k) {
        n_old += (nb[k] == q);
        n_new += (nb[k] == qt);
    }
    int dE = n_old - n_new;
    double dHe = 0.0;
    if (elastic == ORC_ELASTIC_TRACTION)
        dHe = lambda * orc_point_zone_shift(Stab + 36 * (int64_t)q, Stab + 36 * (int64_t)qt, sig_p);
    else if (elastic == ORC_ELASTIC_STRAIN)
        dHe = lambda * orc_point_strain_shift(Stab + 36 * (int64_t)q, Ctab + 36 * (int64_t)q,
                                              Ctab + 36 * (int64_t)qt, sig_p);
    if (dHe == 0.0) {
        *dH = J * dE;
        if (dE <= 0) return 1;
        return (double)r[1] < orc_accept_threshold(dE, J, kT);
    }
    double H = J * dE + dHe;
    double u01 = ((double)r[1] + 0.5) * (1.0 / 4294967296.0);
    double t = (kT > 0.0) ? -kT * log(u01) : 0.0;
    *dH = H;
    *thresh = t;
    return H <= t;
}

/* The same trial with the stress taken from a whole field (N x 6). */
int orc_site_trial(int nx, int ny, int nz, const uint16_t *spin, int x, int y, int z,
                   uint64_t seed, uint32_t mcs, uint32_t replica, double J, double kT,
                   int trial_mode, int Q, int elastic, double lambda, const double *Stab,
                   const double *Ctab, const double *sig, uint16_t *q_new, double *dH, double *thresh)
{
    int64_t p = (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
    return orc_site_trial_at(nx, ny, nz, spin, x, y, z, seed, mcs, replica, J, kT, trial_mode, Q, elastic,
                             lambda, Stab, Ctab, elastic ? sig + 6 * p : NULL, q_new, dH, thresh);
}

/* Red/black half sweep (Sec. "Microstructural Evolution"): every site of one
 * colour, (x+y+z) even = red = 0, is tried against the spins as they were at
 * the start of the half step; same-colour sites have no common neighbour, so
 * updating in place is the same.  Optional per-site outputs (natural order,
 * only this colour's sites written): changed flag, dH and threshold. */
int64_t orc_half_sweep(int nx, int ny, int nz, uint16_t *spin, int colour, uint64_t seed,
                       uint32_t mcs, uint32_t replica, double J, double kT, int trial_mode, int Q,
                       int elastic, double lambda, const double *Stab, const double *Ctab, const double *sig,
                       uint8_t *changed, double *dH_out, double *thresh_out)
{
    int64_t accepted = 0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                if (((x + y + z) & 1) != colour) continue;
                int64_t p = (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
                uint16_t qn;
                double dH, t;
                int acc = orc_site_trial(nx, ny, nz, spin, x, y, z, seed, mcs, replica, J, kT, trial_mode,
                                         Q, elastic, lambda, Stab, Ctab, sig, &qn, &dH, &t);
                if (changed) changed[p] = (uint8_t)acc;
                if (dH_out) dH_out[p] = dH;
                if (thresh_out) thresh_out[p] = t;
                if (acc) {
                    spin[p] = qn;
                    ++accepted;
                }
            }
    return accepted;
}

/* ------------------------------------------------------------------------- */
/* Statistics.                                                                */
/* ------------------------------------------------------------------------- */

/* Number of unlike nearest-neighbour bonds, each bond counted once. */
int64_t orc_unlike_bonds(int nx, int ny, int nz, const uint16_t *spin)
{
    int64_t n = 0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                uint16_t q = spin[x + (int64_t)nx * (y + (int64_t)ny * z)];
                n += q != spin[wrap(x + 1, nx) + (int64_t)nx * (y + (int64_t)ny * z)];
                n += q != spin[x + (int64_t)nx * (wrap(y + 1, ny) + (int64_t)ny * z)];
                n += q != spin[x + (int64_t)nx * (y + (int64_t)ny * wrap(z + 1, nz))];
            }
    return n;
}

/* Volume (site count) of every orientation. */
void orc_orientation_counts(int64_t N, const uint16_t *spin, int Q, int64_t *counts)
{
    memset(counts, 0, sizeof(int64_t) * Q);
    for (int64_t p = 0; p < N; ++p) counts[spin[p]] += 1;
}

/* Gauss-Seidel Monte Carlo step (Sec. "Microstructural Evolution"): N = nx ny nz
 * trials in sequence, each at a site drawn uniformly, each accepted trial applied
 * at once so that later trials see it.  Pure Potts energy (Eq. 4) and Metropolis
 * rule (Eq. 5) with the integer thresholds.  Trial t draws Philox4x32-10 with
 * counter (t, mcs, replica, 1) and key (seed lo, seed hi): word 0 picks the site
 * floor(r0 N / 2^32), word 1 the trial orientation (neighbour k = floor(6 r1 / 2^32)
 * in the order -x,+x,-y,+y,-z,+z, or floor(r1 Q / 2^32)), word 2 the acceptance.
 * Returns the accepted count; *dE_sum (optional) receives the summed bond-count
 * change of the accepted trials. */
int64_t orc_gs_sweep(int nx, int ny, int nz, uint16_t *spin, uint64_t seed, uint32_t mcs, uint32_t replica,
                     double J, double kT, int trial_mode, int Q, int64_t *dE_sum)
{
    const int64_t N = (int64_t)nx * ny * nz;
    const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    int64_t accepted = 0, esum = 0;
    for (int64_t t = 0; t < N; ++t) {
        uint32_t ctr[4] = {(uint32_t)t, mcs, replica, 1u};
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        const int64_t p = (int64_t)(((uint64_t)r[0] * (uint64_t)N) >> 32);
        const int x = (int)(p % nx), y = (int)((p / nx) % ny), z = (int)(p / ((int64_t)nx * ny));
        uint16_t nb[6];
        nb[0] = spin[wrap(x - 1, nx) + (int64_t)nx * (y + (int64_t)ny * z)];
        nb[1] = spin[wrap(x + 1, nx) + (int64_t)nx * (y + (int64_t)ny * z)];
        nb[2] = spin[x + (int64_t)nx * (wrap(y - 1, ny) + (int64_t)ny * z)];
        nb[3] = spin[x + (int64_t)nx * (wrap(y + 1, ny) + (int64_t)ny * z)];
        nb[4] = spin[x + (int64_t)nx * (y + (int64_t)ny * wrap(z - 1, nz))];
        nb[5] = spin[x + (int64_t)nx * (y + (int64_t)ny * wrap(z + 1, nz))];
        const uint16_t q = spin[p];
        const uint16_t qt = trial_mode == ORC_TRIAL_NEIGHBOR ? nb[(int)(((uint64_t)r[1] * 6u) >> 32)]
                                                            : (uint16_t)(((uint64_t)r[1] * (uint64_t)Q) >> 32);
        if (qt == q) continue;
        int dE = 0;
        for (int k = 0; k < 6; ++k) dE += (nb[k] == q) - (nb[k] == qt);
        if (dE <= 0 || (double)r[2] < orc_accept_threshold(dE, J, kT)) {
            spin[p] = qt;
            ++accepted;
            esum += dE;
        }
    }
    if (dE_sum) *dE_sum = esum;
    return accepted;
}

/* Number of grains: connected sets of sites of one orientation, face neighbours
 * (6-connectivity) on the periodic lattice, by breadth-first search.  label
 * (optional, N entries) receives each site's grain index in order of discovery. */
int64_t orc_grain_count(int nx, int ny, int nz, const uint16_t *spin, int64_t *label)
{
    const int64_t N = (int64_t)nx * ny * nz;
    int64_t *lab = label ? label : (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    if (!lab || !queue) {
        if (!label) free(lab);
        free(queue);
        return -1;
    }
    for (int64_t p = 0; p < N; ++p) lab[p] = -1;
    int64_t grains = 0;
    for (int64_t s = 0; s < N; ++s) {
        if (lab[s] >= 0) continue;
        int64_t head = 0, tail = 0;
        queue[tail++] = s;
        lab[s] = grains;
        while (head < tail) {
            const int64_t p = queue[head++];
            const int x = (int)(p % nx), y = (int)((p / nx) % ny), z = (int)(p / ((int64_t)nx * ny));
            const int64_t nbr[6] = {wrap(x - 1, nx) + (int64_t)nx * (y + (int64_t)ny * z),
                                    wrap(x + 1, nx) + (int64_t)nx * (y + (int64_t)ny * z),
                                    x + (int64_t)nx * (wrap(y - 1, ny) + (int64_t)ny * z),
                                    x + (int64_t)nx * (wrap(y + 1, ny) + (int64_t)ny * z),
                                    x + (int64_t)nx * (y + (int64_t)ny * wrap(z - 1, nz)),
                                    x + (int64_t)nx * (y + (int64_t)ny * wrap(z + 1, nz))};
            for (int k = 0; k < 6; ++k)
                if (lab[nbr[k]] < 0 && spin[nbr[k]] == spin[s]) {
                    lab[nbr[k]] = grains;
                    queue[tail++] = nbr[k];
                }
        }
        ++grains;
    }
    if (!label) free(lab);
    free(queue);
    return grains;
}
