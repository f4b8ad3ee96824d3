/*
 * Plain FP64 CPU oracle for the parallel step-wise pulling protocol (PPP).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header or constant table with the CUDA path under
 * paper_1105_4840_gb300/csrc: both sides are written independently from the
 * paper (and from the published definition of Philox4x32-10) and meet only
 * through the seeded synthetic inputs.
 *
 * What it computes, with the passage it follows:
 *   - Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11), uniforms
 *     u = (b + 1/2) 2^-32 and Box-Muller normals.
 *   - The restrained system H(lambda, x) = H_o + k/2 (x - lambda)^2 of
 *     Sec. II, Eq. (3): a synthetic bead chain standing in for deca-alanine
 *     (Sec. IV) with x = |r_{N-1} - r_0| (end-to-end distance), and a 1D
 *     double well U(x) = a (x^2 - 1)^2.
 *   - Restrained Langevin sampling per pulling window (Sec. III (ii), PPP:
 *     every window starts from the same state x_o): BAOAB for the chain,
 *     overdamped Euler-Maruyama for the 1D model; x recorded every `stride`
 *     steps after `n_equil` steps (Sec. IV A records x every 0.1 ps).
 *
 * Everything is FP64 and written for clarity, not speed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Philox4x32-10                                                        */
/* ------------------------------------------------------------------ */

/* One Philox4x32 run of 10 rounds on counter c with key k (SC'11, Sec. 3.3:
 * S-box = two 32x32->64 multiplications, P-box = word permutation, Weyl key
 * schedule with the golden-ratio and sqrt(3)-1 increments). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Four standard normals from one Philox block with counter
 * (c0, c1, c2, c3) and key (seed_lo, seed_hi):  u_m = (b_m + 1/2) 2^-32,
 * n0 = sqrt(-2 ln u0) cos(2 pi u1), n1 = sqrt(-2 ln u0) sin(2 pi u1),
 * n2, n3 likewise from (u2, u3). */
void orc_normals4(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double n[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t b[4];
    orc_philox4x32_10(ctr, key, b);
    double u[4];
    for (int m = 0; m < 4; ++m) u[m] = ((double)b[m] + 0.5) / 4294967296.0;
    double r0 = sqrt(-2.0 * log(u[0]));
    double r1 = sqrt(-2.0 * log(u[2]));
    n[0] = r0 * cos(2.0 * ORC_PI * u[1]);
    n[1] = r0 * sin(2.0 * ORC_PI * u[1]);
    n[2] = r1 * cos(2.0 * ORC_PI * u[3]);
    n[3] = r1 * sin(2.0 * ORC_PI * u[3]);
}

/* Bulk form used by tests: n blocks with counters (c0 + i, c1, c2, c3). */
void orc_philox_bulk(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                     long n, uint32_t *raw, double *normals)
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (long i = 0; i < n; ++i) {
        uint32_t ctr[4] = {c0 + (uint32_t)i, c1, c2, c3};
        if (raw) orc_philox4x32_10(ctr, key, raw + 4 * i);
        if (normals) orc_normals4(seed, c0 + (uint32_t)i, c1, c2, c3, normals + 4 * i);
    }
}

/* Stream tags carried in the fourth counter word. */
enum { ORC_TAG_OSTEP = 0, ORC_TAG_INITVEL = 1 };

/* ------------------------------------------------------------------ */
/* Chain system                                                         */
/* ------------------------------------------------------------------ */

typedef struct {
    int n;                 /* number of beads N                                 */
    const double *sigma;   /* [N] LJ sigma_i (nm)                                */
    const double *eps;     /* [N] LJ epsilon_i (kJ/mol)                          */
    const double *q;       /* [N] charge (e)                                     */
    const double *mass;    /* [N] mass (amu)                                     */
    double kb, r0;         /* bond U = kb/2 (r - r0)^2 for (i, i+1)              */
    double ktheta, theta0; /* angle U = ktheta/2 (theta - theta0)^2, (i,i+1,i+2) */
    const double *dih_k;   /* [N][3] K_n of the dihedral starting at bead i      */
    const double *dih_phase; /* [N][3] delta_n of that dihedral (radians)        */
    double ke;             /* Coulomb constant (kJ mol^-1 nm e^-2)               */
    int nonbonded;         /* 0: no LJ / Coulomb terms at all                    */
} orc_chain;

static inline void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static inline double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* Dihedral angle of beads a-b-c-d, IUPAC convention:
 * phi = atan2(|b2| b1 . (b2 x b3), (b1 x b2) . (b2 x b3)). */
static double dihedral_angle(const double *ra, const double *rb, const double *rc, const double *rd)
{
    double b1[3], b2[3], b3[3], n1[3], n2[3];
    sub3(rb, ra, b1); sub3(rc, rb, b2); sub3(rd, rc, b3);
    cross3(b1, b2, n1); cross3(b2, b3, n2);
    return atan2(norm3(b2) * dot3(b1, n2), dot3(n1, n2));
}

static double bond_angle(const double *ra, const double *rb, const double *rc)
{
    double u[3], w[3];
    sub3(ra, rb, u); sub3(rc, rb, w);
    double c = dot3(u, w) / (norm3(u) * norm3(w));
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    return acos(c);
}

/* Total potential energy of the restrained chain, H(lambda, x) of Eq. (3)
 * without momenta.  parts (optional, 6 doubles): bond, angle, dihedral,
 * Lennard-Jones, Coulomb, trap. */
double orc_chain_energy(const orc_chain *c, const double *r, double lambda, double k, double *parts)
{
    const int n = c->n;
    double eb = 0, ea = 0, ed = 0, elj = 0, eq = 0, et = 0;
    for (int i = 0; i + 1 < n; ++i) {
        double d[3];
        sub3(r + 3 * (i + 1), r + 3 * i, d);
        double len = norm3(d);
        eb += 0.5 * c->kb * (len - c->r0) * (len - c->r0);
    }
    for (int i = 0; c->ktheta != 0.0 && i + 2 < n; ++i) {
        double th = bond_angle(r + 3 * i, r + 3 * (i + 1), r + 3 * (i + 2));
        ea += 0.5 * c->ktheta * (th - c->theta0) * (th - c->theta0);
    }
    for (int i = 0; i + 3 < n; ++i) {
        if (c->dih_k[3 * i] == 0.0 && c->dih_k[3 * i + 1] == 0.0 && c->dih_k[3 * i + 2] == 0.0) continue;
        double phi = dihedral_angle(r + 3 * i, r + 3 * (i + 1), r + 3 * (i + 2), r + 3 * (i + 3));
        for (int m = 0; m < 3; ++m)
            ed += c->dih_k[3 * i + m] * (1.0 + cos((m + 1) * phi - c->dih_phase[3 * i + m]));
    }
    if (c->nonbonded) {
        for (int i = 0; i < n; ++i)
            for (int j = i + 3; j < n; ++j) {
                double d[3];
                sub3(r + 3 * j, r + 3 * i, d);
                double rr = norm3(d);
                double sij = 0.5 * (c->sigma[i] + c->sigma[j]);
                double eij = sqrt(c->eps[i] * c->eps[j]);
                double sr2 = (sij / rr) * (sij / rr);
                double sr6 = sr2 * sr2 * sr2;
                elj += 4.0 * eij * (sr6 * sr6 - sr6);
                eq += c->ke * c->q[i] * c->q[j] / rr;
            }
    }
    {
        double d[3];
        sub3(r + 3 * (n - 1), r, d);
        double x = norm3(d);
        et = 0.5 * k * (x - lambda) * (x - lambda);
    }
    if (parts) { parts[0] = eb; parts[1] = ea; parts[2] = ed; parts[3] = elj; parts[4] = eq; parts[5] = et; }
    return eb + ea + ed + elj + eq + et;
}

/* Reaction coordinate x = |r_{N-1} - r_0|. */
double orc_chain_rc(const orc_chain *c, const double *r)
{
    double d[3];
    sub3(r + 3 * (c->n - 1), r, d);
    return norm3(d);
}

/* Analytic forces F = -grad H(lambda, x). */
void orc_chain_forces(const orc_chain *c, const double *r, double lambda, double k, double *f)
{
    const int n = c->n;
    memset(f, 0, sizeof(double) * 3 * (size_t)n);
    /* bonds */
    for (int i = 0; i + 1 < n; ++i) {
        double d[3];
        sub3(r + 3 * (i + 1), r + 3 * i, d);
        double len = norm3(d);
        double g = c->kb * (len - c->r0) / len; /* dU/dr / r */
        for (int a = 0; a < 3; ++a) {
            f[3 * i + a] += g * d[a];
            f[3 * (i + 1) + a] -= g * d[a];
        }
    }
    /* angles: dU/dtheta * dtheta/dr with dtheta = -dcos / sin(theta) */
    for (int i = 0; c->ktheta != 0.0 && i + 2 < n; ++i) {
        const double *ra = r + 3 * i, *rb = r + 3 * (i + 1), *rc = r + 3 * (i + 2);
        double u[3], w[3];
        sub3(ra, rb, u); sub3(rc, rb, w);
        double lu = norm3(u), lw = norm3(w);
        double cs = dot3(u, w) / (lu * lw);
        if (cs > 1.0) cs = 1.0;
        if (cs < -1.0) cs = -1.0;
        double th = acos(cs);
        double sn = sqrt(1.0 - cs * cs);
        double dudth = c->ktheta * (th - c->theta0);
        double pref = dudth / sn; /* F = pref * dcos/dr */
        double ga[3], gc[3];
        for (int a = 0; a < 3; ++a) {
            ga[a] = w[a] / (lu * lw) - cs * u[a] / (lu * lu);
            gc[a] = u[a] / (lu * lw) - cs * w[a] / (lw * lw);
        }
        for (int a = 0; a < 3; ++a) {
            f[3 * i + a] += pref * ga[a];
            f[3 * (i + 2) + a] += pref * gc[a];
            f[3 * (i + 1) + a] -= pref * (ga[a] + gc[a]);
        }
    }
    /* dihedrals: dU/dphi * dphi/dr (Blondel & Karplus gradient of the IUPAC angle) */
    for (int i = 0; i + 3 < n; ++i) {
        if (c->dih_k[3 * i] == 0.0 && c->dih_k[3 * i + 1] == 0.0 && c->dih_k[3 * i + 2] == 0.0) continue;
        const double *ra = r + 3 * i, *rb = r + 3 * (i + 1), *rc = r + 3 * (i + 2), *rd = r + 3 * (i + 3);
        double b1[3], b2[3], b3[3], n1[3], n2[3];
        sub3(rb, ra, b1); sub3(rc, rb, b2); sub3(rd, rc, b3);
        cross3(b1, b2, n1); cross3(b2, b3, n2);
        double phi = atan2(norm3(b2) * dot3(b1, n2), dot3(n1, n2));
        double dudphi = 0.0;
        for (int m = 0; m < 3; ++m)
            dudphi -= (m + 1) * c->dih_k[3 * i + m] * sin((m + 1) * phi - c->dih_phase[3 * i + m]);
        double lb2 = norm3(b2);
        double nn1 = dot3(n1, n1), nn2 = dot3(n2, n2);
        double ga[3], gd[3], gb[3], gc[3];
        double p = dot3(b1, b2) / (lb2 * lb2), q = dot3(b3, b2) / (lb2 * lb2);
        for (int a = 0; a < 3; ++a) {
            ga[a] = -lb2 / nn1 * n1[a];
            gd[a] = lb2 / nn2 * n2[a];
        }
        for (int a = 0; a < 3; ++a) {
            gb[a] = -(1.0 + p) * ga[a] + q * gd[a];
            gc[a] = -(1.0 + q) * gd[a] + p * ga[a];
        }
        for (int a = 0; a < 3; ++a) {
            f[3 * i + a] -= dudphi * ga[a];
            f[3 * (i + 1) + a] -= dudphi * gb[a];
            f[3 * (i + 2) + a] -= dudphi * gc[a];
            f[3 * (i + 3) + a] -= dudphi * gd[a];
        }
    }
    /* nonbonded: all pairs with j - i >= 3 */
    if (c->nonbonded) {
        for (int i = 0; i < n; ++i)
            for (int j = i + 3; j < n; ++j) {
                double d[3];
                sub3(r + 3 * j, r + 3 * i, d);
                double rr = norm3(d);
                double sij = 0.5 * (c->sigma[i] + c->sigma[j]);
                double eij = sqrt(c->eps[i] * c->eps[j]);
                double sr2 = (sij / rr) * (sij / rr);
                double sr6 = sr2 * sr2 * sr2;
                /* dU/dr = -(24 eps (2 sr12 - sr6) + ke qi qj / r) / r */
                double dudr = -(24.0 * eij * (2.0 * sr6 * sr6 - sr6) + c->ke * c->q[i] * c->q[j] / rr) / rr;
                for (int a = 0; a < 3; ++a) {
                    double fa = dudr * d[a] / rr; /* gradient wrt r_j */
                    f[3 * j + a] -= fa;
                    f[3 * i + a] += fa;
                }
            }
    }
    /* trap on x = |r_{N-1} - r_0| */
    {
        double d[3];
        sub3(r + 3 * (n - 1), r, d);
        double x = norm3(d);
        double g = k * (x - lambda) / x;
        for (int a = 0; a < 3; ++a) {
            f[3 * (n - 1) + a] -= g * d[a];
            f[a] += g * d[a];
        }
    }
}

/* Standard normals for the 3N degrees of freedom of one replica at one
 * step: block b of Philox counter (b, uid, step, tag) supplies the normals of
 * dofs 4b .. 4b+3, dof d = 3 * bead + axis.  xi must hold 4 ceil(3N/4). */
static void dof_normals(int n, uint64_t seed, uint32_t uid, uint32_t step, uint32_t tag, double *xi)
{
    const int nblk = (3 * n + 3) / 4;
    for (int b = 0; b < nblk; ++b) orc_normals4(seed, (uint32_t)b, uid, step, tag, xi + 4 * b);
}

/* Maxwell-Boltzmann velocities: v = sqrt(kT/m) * xi with the dof normals of
 * step 0 and tag TAG_INITVEL. */
void orc_chain_init_velocities(const orc_chain *c, double kT, uint64_t seed, uint32_t uid, double *v)
{
    double *xi = (double *)malloc(sizeof(double) * 4 * (size_t)((3 * c->n + 3) / 4));
    if (!xi) return;
    dof_normals(c->n, seed, uid, 0u, ORC_TAG_INITVEL, xi);
    for (int i = 0; i < c->n; ++i) {
        double s = sqrt(kT / c->mass[i]);
        for (int a = 0; a < 3; ++a) v[3 * i + a] = s * xi[3 * i + a];
    }
    free(xi);
}

/* BAOAB Langevin integration of one replica in one window.
 *   per step n:  v += dt/2 F/m;  r += dt/2 v;
 *                v = c1 v + c2 sqrt(kT/m) xi_n   (dof normals of step n, TAG_OSTEP);
 *                r += dt/2 v;  F = F(r);  v += dt/2 F/m
 * with c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2).  After step n (1-based
 * count n+1 > n_equil with (n+1-n_equil) % stride == 0) x = |r_{N-1}-r_0| is
 * stored.  r, v are read as the start state and overwritten with the final
 * state.  If init_v != 0 velocities are drawn first.  Returns the number of
 * samples written, or -1 if a coordinate became non-finite. */
long orc_chain_run_from(const orc_chain *c, double lambda, double k, double kT, double dt, double gamma,
                        long step0, long n_steps, long n_equil, long stride, uint64_t seed, uint32_t uid,
                        double *r, double *v, int init_v, double *samples);

long orc_chain_run(const orc_chain *c, double lambda, double k, double kT, double dt, double gamma,
                   long n_steps, long n_equil, long stride, uint64_t seed, uint32_t uid,
                   double *r, double *v, int init_v, double *samples)
{
    return orc_chain_run_from(c, lambda, k, kT, dt, gamma, 0, n_steps, n_equil, stride, seed, uid, r, v, init_v,
                              samples);
}

/* As orc_chain_run, with the time steps numbered step0 .. step0 + n_steps - 1
 * for the O-step noise (counter (block, uid, step, 0)); equilibration and
 * sampling count from the first of them.  The sequential pulling protocol
 * (Sec. III (i)) runs window i with step0 = i * tau from the state window
 * i - 1 left. */
long orc_chain_run_from(const orc_chain *c, double lambda, double k, double kT, double dt, double gamma,
                        long step0, long n_steps, long n_equil, long stride, uint64_t seed, uint32_t uid,
                        double *r, double *v, int init_v, double *samples)
{
    const int n = c->n;
    double *f = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *xi = (double *)malloc(sizeof(double) * 4 * (size_t)((3 * n + 3) / 4));
    if (!f || !xi) { free(f); free(xi); return -1; }
    if (init_v) orc_chain_init_velocities(c, kT, seed, uid, v);
    const double c1 = exp(-gamma * dt);
    const double c2 = sqrt(1.0 - c1 * c1);
    orc_chain_forces(c, r, lambda, k, f);
    long ns = 0;
    for (long step = 0; step < n_steps; ++step) {
        dof_normals(n, seed, uid, (uint32_t)(step0 + step), ORC_TAG_OSTEP, xi);
        for (int i = 0; i < n; ++i) {
            double im = 1.0 / c->mass[i];
            double sv = sqrt(kT * im);
            for (int a = 0; a < 3; ++a) {
                double *vv = v + 3 * i + a, *rr = r + 3 * i + a;
                *vv += 0.5 * dt * f[3 * i + a] * im;
                *rr += 0.5 * dt * (*vv);
                *vv = c1 * (*vv) + c2 * sv * xi[3 * i + a];
                *rr += 0.5 * dt * (*vv);
            }
        }
        orc_chain_forces(c, r, lambda, k, f);
        for (int i = 0; i < n; ++i) {
            double im = 1.0 / c->mass[i];
            for (int a = 0; a < 3; ++a) v[3 * i + a] += 0.5 * dt * f[3 * i + a] * im;
        }
        long done = step + 1;
        if (done > n_equil && (done - n_equil) % stride == 0) samples[ns++] = orc_chain_rc(c, r);
        if (!isfinite(r[0]) || !isfinite(r[3 * (n - 1)])) { free(f); free(xi); return -1; }
    }
    free(f);
    free(xi);
    return ns;
}

/* Constant-velocity pulling (the steered-MD comparator of Sec. I): n_equil
 * BAOAB steps with the trap at lambda1, then the trap centre advances by
 * vdt per step: at the force evaluation that ends step n (time n + 1) it
 * sits at lambda(n + 1) = lambda1 + vdt (n + 1 - n_equil) for n + 1 > n_equil,
 * and the move from lambda(n) to lambda(n + 1) does the work of Eq. (9) at
 * the reaction coordinate of that moment,
 *   k/2 (lambda(n+1) - lambda(n)) (lambda(n+1) + lambda(n) - 2 x),
 * the discrete form of -v k int (x - lambda1 - v t) dt.  Every `stride` steps
 * of pulling, x and the accumulated work are recorded. */
long orc_chain_smd(const orc_chain *c, double lambda1, double vdt, double k, double kT, double dt, double gamma,
                   long n_steps, long n_equil, long stride, uint64_t seed, uint32_t uid,
                   double *r, double *v, double *x_out, double *w_out)
{
    const int n = c->n;
    double *f = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *xi = (double *)malloc(sizeof(double) * 4 * (size_t)((3 * n + 3) / 4));
    if (!f || !xi) { free(f); free(xi); return -1; }
    orc_chain_init_velocities(c, kT, seed, uid, v);
    const double c1 = exp(-gamma * dt);
    const double c2 = sqrt(1.0 - c1 * c1);
    double lam = lambda1, work = 0.0;
    orc_chain_forces(c, r, lam, k, f);
    long ns = 0;
    for (long step = 0; step < n_steps; ++step) {
        dof_normals(n, seed, uid, (uint32_t)step, ORC_TAG_OSTEP, xi);
        for (int i = 0; i < n; ++i) {
            double im = 1.0 / c->mass[i];
            double sv = sqrt(kT * im);
            for (int a = 0; a < 3; ++a) {
                double *vv = v + 3 * i + a, *rr = r + 3 * i + a;
                *vv += 0.5 * dt * f[3 * i + a] * im;
                *rr += 0.5 * dt * (*vv);
                *vv = c1 * (*vv) + c2 * sv * xi[3 * i + a];
                *rr += 0.5 * dt * (*vv);
            }
        }
        const long done = step + 1;
        if (done > n_equil) {
            const double lam_new = lambda1 + vdt * (double)(done - n_equil);
            const double x = orc_chain_rc(c, r);
            work += 0.5 * k * (lam_new - lam) * (lam_new + lam - 2.0 * x);
            lam = lam_new;
        }
        orc_chain_forces(c, r, lam, k, f);
        for (int i = 0; i < n; ++i) {
            double im = 1.0 / c->mass[i];
            for (int a = 0; a < 3; ++a) v[3 * i + a] += 0.5 * dt * f[3 * i + a] * im;
        }
        if (done > n_equil && (done - n_equil) % stride == 0) {
            x_out[ns] = orc_chain_rc(c, r);
            w_out[ns] = work;
            ++ns;
        }
        if (!isfinite(r[0]) || !isfinite(r[3 * (n - 1)])) { free(f); free(xi); return -1; }
    }
    free(f);
    free(xi);
    return ns;
}

/* Kinetic energy sum m v^2 / 2. */
double orc_chain_kinetic(const orc_chain *c, const double *v)
{
    double e = 0;
    for (int i = 0; i < c->n; ++i) e += 0.5 * c->mass[i] * dot3(v + 3 * i, v + 3 * i);
    return e;
}

/* ------------------------------------------------------------------ */
/* 1D model                                                             */
/* ------------------------------------------------------------------ */

double orc_od1d_force(double a, double lambda, double k, double x);

/* Constant-velocity pulling of the 1D model: step n moves x with the trap at
 * lambda(n) = lambda1 + vdt max(0, n - n_equil); before step n (n > n_equil)
 * the trap moves from lambda(n - 1) with the work of Eq. (9) at the current
 * x.  Records x and the accumulated work every `stride` steps of pulling. */
long orc_od1d_smd(double a, double lambda1, double vdt, double k, double kT, double gamma, double dt,
                  long n_steps, long n_equil, long stride, uint64_t seed, uint32_t uid, double x0,
                  double *x_out, double *w_out)
{
    double x = x0, lam = lambda1, work = 0.0;
    double xi[4] = {0, 0, 0, 0};
    const double amp = sqrt(2.0 * kT * dt / gamma);
    long ns = 0;
    for (long step = 0; step < n_steps; ++step) {
        if (step > n_equil) {
            const double lam_new = lambda1 + vdt * (double)(step - n_equil);
            work += 0.5 * k * (lam_new - lam) * (lam_new + lam - 2.0 * x);
            lam = lam_new;
        }
        if ((step & 3) == 0) orc_normals4(seed, 0u, uid, (uint32_t)(step >> 2), ORC_TAG_OSTEP, xi);
        x = x + orc_od1d_force(a, lam, k, x) * dt / gamma + amp * xi[step & 3];
        const long done = step + 1;
        if (done > n_equil && (done - n_equil) % stride == 0) {
            x_out[ns] = x;
            w_out[ns] = work;
            ++ns;
        }
    }
    return ns;
}

/* Force of U(x) = a (x^2 - 1)^2 plus the trap k/2 (x - lambda)^2. */
double orc_od1d_force(double a, double lambda, double k, double x)
{
    return -4.0 * a * x * (x * x - 1.0) - k * (x - lambda);
}

/* Overdamped Euler-Maruyama with friction gamma:
 *   x_{n+1} = x_n + F(x_n) dt / gamma + sqrt(2 kT dt / gamma) xi_n,
 * xi_n = normal (n mod 4) of the Philox block (0, uid, n div 4, TAG_OSTEP).
 * Sampling schedule as in orc_chain_run.  Returns the sample count. */
long orc_od1d_run_from(double a, double lambda, double k, double kT, double gamma, double dt, long step0,
                       long n_steps, long n_equil, long stride, uint64_t seed, uint32_t uid,
                       double x0, double *samples, double *x_final);

long orc_od1d_run(double a, double lambda, double k, double kT, double gamma, double dt,
                  long n_steps, long n_equil, long stride, uint64_t seed, uint32_t uid,
                  double x0, double *samples, double *x_final)
{
    return orc_od1d_run_from(a, lambda, k, kT, gamma, dt, 0, n_steps, n_equil, stride, seed, uid, x0, samples,
                             x_final);
}

/* As orc_od1d_run with the steps numbered step0 .. step0 + n_steps - 1 for
 * the noise (normal n mod 4 of block (0, uid, n div 4, 0)). */
long orc_od1d_run_from(double a, double lambda, double k, double kT, double gamma, double dt, long step0,
                       long n_steps, long n_equil, long stride, uint64_t seed, uint32_t uid,
                       double x0, double *samples, double *x_final)
{
    double x = x0;
    double xi[4] = {0, 0, 0, 0};
    const double amp = sqrt(2.0 * kT * dt / gamma);
    long ns = 0;
    for (long step = 0; step < n_steps; ++step) {
        const long n = step0 + step;
        if ((n & 3) == 0 || step == 0) orc_normals4(seed, 0u, uid, (uint32_t)(n >> 2), ORC_TAG_OSTEP, xi);
        x = x + orc_od1d_force(a, lambda, k, x) * dt / gamma + amp * xi[n & 3];
        long done = step + 1;
        if (done > n_equil && (done - n_equil) % stride == 0) samples[ns++] = x;
    }
    if (x_final) *x_final = x;
    return ns;
}
