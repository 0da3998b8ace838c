/*
 * ptca_oracle.c -- plain, slow, FP64 CPU oracle for the traveling-cluster
 * Monte Carlo hot path (TCA, Sec. II; its parallel reorganisation PTCA, Sec. III).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or helper with
 * the CUDA path; the two implement the same published definitions
 * independently (including the Philox4x32-10 counter generator).
 *
 * Everything is written for obviousness, not speed:
 *   - the cluster Hamiltonian is built as a dense n x n complex matrix;
 *   - eigenvalues come from a cyclic complex Jacobi method applied to the whole
 *     matrix (no tridiagonalisation, no blocking);
 *   - a sweep visits the sites one at a time in the flattened stage order and
 *     each visit reads the CURRENT spins (sequential TCA, Sec. II.c steps a-f),
 *     so it makes no use of the independence that PTCA exploits.
 *
 * Build without fast-math and without FMA contraction so that the results are
 * the same on x86-64 and aarch64:
 *     gcc -O2 -std=c11 -fPIC -shared -ffp-contract=off -o libptca_oracle.so ptca_oracle.c -lm
 *
 * Models on a chain, a square or a cubic lattice, all with hopping -t between
 * nearest neighbours of the same spin and two rows per cluster site in the
 * cluster matrix (two spin species; Sec. IV gives the order as twice the
 * cluster sites):
 *   model 0, double exchange: a Hund term -J_H S_i . sigma on every site, with
 *     classical unit spins S_i;
 *   model 1, Hubbard mean field (Eq. 1, <n_i> = 1): an on-site term
 *     (U/2)(n_i - m_i . sigma_i) with classical vectors m_i of any length, and
 *     the classical energy (U/4)(m_i^2 - 1) of every site, which the cluster
 *     free energy includes for the sites of its window;
 *   model 2, adiabatic Holstein (the model of Sec. VII.b): a classical
 *     distortion x_i per site (component 0 of the site's vector; the other
 *     two stay 0), the one-body term lambda x_i n_i, and the classical energy
 *     K/2 x_i^2 - lambda x_i + mu of every window site (the rest of
 *     (lambda x_i - mu)(n_i - 1) + K/2 x_i^2; -mu n_i is the chemical
 *     potential of the free energy).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const double PI = 3.14159265358979323846;

/* Parameters of one oracle problem.  The field layout is mirrored by the
 * ctypes wrapper in oracle/__init__.py and by nothing else. */
typedef struct {
    int32_t Lx, Ly;            /* lattice extents; Ly == 1 means a 1-D chain      */
                               /* (Lz, the third extent, is the last field)       */
    int32_t lattice_periodic;  /* 1: torus, 0: open edges                         */
    int32_t Lc;                /* linear cluster size L_c (N_c = L_c^2 in 2-D)    */
    int32_t ox, oy;            /* position of the update site inside the window  */
    int32_t cluster_periodic;  /* 1: periodic wrap inside the window, 0: open    */
    int32_t schedule;          /* 0: tiled sublattice, 1: 2^d blocks (Sec. III.a) */
    int32_t stride;            /* tiled schedule: centre spacing                 */
    int32_t proposal;          /* 0: uniform on the sphere, 1: cone around S_old */
    double t, JH, mu, T;
    double cone_deg;
    uint64_t seed;
    int32_t model;             /* 0: double exchange, 1: Hubbard mean field      */
    int32_t pad0;
    double U;                  /* model 1: Hubbard U                             */
    double m_step;             /* model 1: radius of the proposal ball           */
    int32_t Lz;                /* third extent; 1 for a square lattice or chain  */
    int32_t oz;                /* update-site position along z                    */
    double lam;                /* model 2: electron-lattice coupling lambda      */
    double K;                  /* model 2: elastic constant                      */
} oracle_model;

/* Sites: index (z Ly + y) Lx + x.  Lz > 1 needs Ly > 1 (cubic lattice). */
static int n_sites(const oracle_model* m) { return m->Lx * m->Ly * m->Lz; }
static int cluster_dim(const oracle_model* m) { return 1 + (m->Ly > 1) + (m->Lz > 1); }
static int n_max(const oracle_model* m)
{
    int ns = 1;
    for (int d = 0; d < cluster_dim(m); ++d) ns *= m->Lc;
    return 2 * ns;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Ten rounds of the 4x32 Philox S-box; the key is */
/* bumped by the Weyl constants between rounds.                              */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t key[2], const uint32_t ctr[4], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t k0 = key[0], k1 = key[1];
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
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

/* Random-number stream of the method: key = seed, counter = (site, purpose,
 * sweep lo, sweep hi).  Two doubles per call, each built from 53 bits of a
 * 64-bit word as (x/2^11 + 1/2) * 2^-53, which lies strictly inside (0,1). */
enum { PURPOSE_INIT = 0, PURPOSE_PROPOSE = 1, PURPOSE_ACCEPT = 2, PURPOSE_RADIUS = 4 };

void oracle_uniform2(uint64_t seed, uint64_t sweep, uint32_t site, uint32_t purpose, double u[2])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {site, purpose, (uint32_t)sweep, (uint32_t)(sweep >> 32)};
    uint32_t w[4];
    oracle_philox4x32_10(key, ctr, w);
    uint64_t xa = ((uint64_t)w[1] << 32) | w[0];
    uint64_t xb = ((uint64_t)w[3] << 32) | w[2];
    u[0] = ((double)(xa >> 11) + 0.5) * 0x1p-53;
    u[1] = ((double)(xb >> 11) + 0.5) * 0x1p-53;
}

/* Unit vector uniform on the sphere from two uniforms: z uniform in (-1,1),
 * azimuth uniform in (0, 2 pi). */
static void sphere_point(const double u[2], double s[3])
{
    double z = 2.0 * u[0] - 1.0;
    double phi = 2.0 * PI * u[1];
    double r = sqrt(fmax(0.0, 1.0 - z * z));
    s[0] = r * cos(phi);
    s[1] = r * sin(phi);
    s[2] = z;
}

/* Initial classical variables: independent unit vectors uniform on the
 * sphere (models 0, 1); distortions x_i uniform in [-1, 1] (model 2). */
void oracle_init_spins(const oracle_model* m, double* S)
{
    int N = n_sites(m);
    for (int i = 0; i < N; ++i) {
        double u[2];
        oracle_uniform2(m->seed, 0, (uint32_t)i, PURPOSE_INIT, u);
        if (m->model == 2) {
            S[3 * i] = 2.0 * u[0] - 1.0;
            S[3 * i + 1] = 0.0;
            S[3 * i + 2] = 0.0;
        } else {
            sphere_point(u, S + 3 * i);
        }
    }
}

/* Proposed new spin at a site (Sec. II.c step c: a random change of the
 * update site's classical variable).  Sphere: a fresh uniform point.  Cone:
 * a point uniform on the spherical cap of half-angle cone_deg around S_old,
 * i.e. cos(theta) uniform in [cos(cone), 1], rotated from the z axis onto
 * S_old.  The Holstein and Hubbard moves are the first two branches. */
void oracle_propose(const oracle_model* m, uint64_t sweep, int site, const double* s_old, double* s_new)
{
    double u[2];
    oracle_uniform2(m->seed, sweep, (uint32_t)site, PURPOSE_PROPOSE, u);
    if (m->model == 2) {
        /* Holstein: x_new = x_old + m_step (2u - 1), uniform in
         * [x_old - m_step, x_old + m_step]; symmetric. */
        s_new[0] = s_old[0] + m->m_step * (2.0 * u[0] - 1.0);
        s_new[1] = s_old[1];
        s_new[2] = s_old[2];
        return;
    }
    if (m->model == 1) {
        /* Hubbard mean field: m_new = m_old + d, d uniform in the ball of
         * radius m_step (direction uniform on the sphere, radius
         * m_step * v^(1/3)).  The proposal is symmetric in (m_old, m_new), so
         * Metropolis on dF samples exp(-F/T) d^3m. */
        double dir[3], v[2];
        sphere_point(u, dir);
        oracle_uniform2(m->seed, sweep, (uint32_t)site, PURPOSE_RADIUS, v);
        double r = m->m_step * cbrt(v[0]);
        for (int k = 0; k < 3; ++k) s_new[k] = s_old[k] + r * dir[k];
        return;
    }
    if (m->proposal == 0) {
        sphere_point(u, s_new);
        return;
    }
    double cmin = cos(m->cone_deg * PI / 180.0);
    double ct = 1.0 - u[0] * (1.0 - cmin);
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double phi = 2.0 * PI * u[1];
    double v[3] = {st * cos(phi), st * sin(phi), ct};
    double a = s_old[0], b = s_old[1], c = s_old[2];
    double r[3];
    if (c < -1.0 + 1e-12) {
        /* S_old is (anti)parallel to -z: rotate by pi about x. */
        r[0] = v[0]; r[1] = -v[1]; r[2] = -v[2];
    } else {
        /* Rotation matrix that maps z onto (a,b,c). */
        double k = 1.0 / (1.0 + c);
        double R00 = 1.0 - a * a * k, R01 = -a * b * k, R02 = a;
        double R10 = -a * b * k, R11 = 1.0 - b * b * k, R12 = b;
        double R20 = -a, R21 = -b, R22 = c;
        r[0] = R00 * v[0] + R01 * v[1] + R02 * v[2];
        r[1] = R10 * v[0] + R11 * v[1] + R12 * v[2];
        r[2] = R20 * v[0] + R21 * v[1] + R22 * v[2];
    }
    double nr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    s_new[0] = r[0] / nr; s_new[1] = r[1] / nr; s_new[2] = r[2] / nr;
}

/* ------------------------------------------------------------------------ */
/* Traveling cluster: window around an update site (Sec. II.b, Fig. 1).     */
/* ------------------------------------------------------------------------ */

/* Window along one axis.  Periodic lattice: L_c consecutive sites starting
 * o before the update site, wrapped modulo L.  Open lattice: the same range
 * clipped to [0, L-1]. */
static void window_axis(int L, int periodic, int Lc, int o, int c, int* start, int* ext)
{
    if (L == 1) { *start = 0; *ext = 1; return; }
    int a = c - o, b = c - o + Lc - 1;
    if (periodic) { *start = ((a % L) + L) % L; *ext = Lc; return; }
    if (a < 0) a = 0;
    if (b > L - 1) b = L - 1;
    *start = a; *ext = b - a + 1;
}

/* The window of an update site: start and extent along each axis. */
typedef struct { int x0, y0, z0, ex, ey, ez; } window;

static window window_of(const oracle_model* m, int site)
{
    window w;
    int cx = site % m->Lx, cy = (site / m->Lx) % m->Ly, cz = site / (m->Lx * m->Ly);
    window_axis(m->Lx, m->lattice_periodic, m->Lc, m->ox, cx, &w.x0, &w.ex);
    window_axis(m->Ly, m->lattice_periodic, m->Lc, m->oy, cy, &w.y0, &w.ey);
    window_axis(m->Lz, m->lattice_periodic, m->Lc, m->oz, cz, &w.z0, &w.ez);
    return w;
}

/* Lattice site at window coordinates (wx, wy, wz). */
static int window_site(const oracle_model* m, const window* w, int wx, int wy, int wz)
{
    int x = w->x0 + wx, y = w->y0 + wy, z = w->z0 + wz;
    if (m->lattice_periodic) { x %= m->Lx; y %= m->Ly; z %= m->Lz; }
    return (z * m->Ly + y) * m->Lx + x;
}

/* Dense cluster Hamiltonian H_clus{C[i_s]} (Sec. II.c step b) for update site
 * `site`.  Basis index 2*((wz*ey + wy)*ex + wx) + spin.  Spin of the update
 * site is replaced by s_new when s_new != NULL (step d).  Returns
 * n = 2*ex*ey*ez and writes H (n*n complex, row-major) and the window extents
 * along x and y.  The cluster boundary is periodic inside the window when
 * m->cluster_periodic (Sec. II.b: periodic boundary conditions on the
 * cluster); an axis of extent 2 then has two bonds between its two sites, an
 * axis of extent 1 has none. */
int oracle_cluster_hamiltonian(const oracle_model* m, const double* S, int site,
                               const double* s_new, cplx* H, int* ex_out, int* ey_out)
{
    window win = window_of(m, site);
    int ex = win.ex, ey = win.ey, ez = win.ez;
    int nsite = ex * ey * ez, n = 2 * nsite;
    memset(H, 0, sizeof(cplx) * (size_t)n * (size_t)n);
    for (int wz = 0; wz < ez; ++wz)
    for (int wy = 0; wy < ey; ++wy) {
        for (int wx = 0; wx < ex; ++wx) {
            int w = (wz * ey + wy) * ex + wx;
            int g = window_site(m, &win, wx, wy, wz);
            const double* s = S + 3 * g;
            if (s_new && g == site) s = s_new;
            /* On-site 2x2 spin block: -J_H S.sigma (model 0),
             * (U/2) 1 - (U/2) m.sigma (model 1), or lambda x 1 (model 2). */
            int a = 2 * w, b = 2 * w + 1;
            double J = m->model == 1 ? 0.5 * m->U : (m->model == 2 ? 0.0 : m->JH);
            double e0 = m->model == 1 ? 0.5 * m->U : (m->model == 2 ? m->lam * s[0] : 0.0);
            H[a * n + a] += e0 - J * s[2];
            H[b * n + b] += e0 + J * s[2];
            H[a * n + b] += -J * (s[0] - I * s[1]);
            H[b * n + a] += -J * (s[0] + I * s[1]);
            /* Hopping -t to the +x, +y and +z neighbours (each bond once). */
            int nb[3] = {-1, -1, -1};
            if (wx + 1 < ex) nb[0] = (wz * ey + wy) * ex + (wx + 1);
            else if (m->cluster_periodic && ex >= 2) nb[0] = (wz * ey + wy) * ex + 0;
            if (wy + 1 < ey) nb[1] = (wz * ey + wy + 1) * ex + wx;
            else if (m->cluster_periodic && ey >= 2) nb[1] = (wz * ey + 0) * ex + wx;
            if (wz + 1 < ez) nb[2] = ((wz + 1) * ey + wy) * ex + wx;
            else if (m->cluster_periodic && ez >= 2) nb[2] = (0 * ey + wy) * ex + wx;
            for (int d = 0; d < 3; ++d) {
                if (nb[d] < 0) continue;
                for (int sp = 0; sp < 2; ++sp) {
                    int i = 2 * w + sp, j = 2 * nb[d] + sp;
                    H[i * n + j] += -m->t;
                    H[j * n + i] += -m->t;
                }
            }
        }
    }
    if (ex_out) *ex_out = ex;
    if (ey_out) *ey_out = ey;
    return n;
}

/* ------------------------------------------------------------------------ */
/* Cyclic Jacobi eigenvalue method for a complex Hermitian matrix.           */
/* Each rotation acts on rows/columns p,q with the unitary                   */
/*     U = [[c, s w], [-s conj(w), c]],  w = A_pq/|A_pq|,                     */
/* t = tan(theta) the smaller root of t^2 + 2 zeta t - 1 = 0,                 */
/* zeta = (A_qq - A_pp)/(2|A_pq|), which zeroes A_pq in U^H A U.  Sweeps     */
/* continue until the off-diagonal Frobenius norm is below 1e-14 ||A||_F.    */
/* A is overwritten; eig receives the eigenvalues in ascending order.         */
/* Returns the number of sweeps, or -1 if 100 sweeps did not converge.        */
/* ------------------------------------------------------------------------ */
static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

int oracle_eigvalsh_jacobi(int n, cplx* A, double* eig)
{
    double fro2 = 0.0;
    for (int i = 0; i < n * n; ++i) fro2 += creal(A[i] * conj(A[i]));
    int sweeps = 0, converged = 0;
    for (; sweeps < 100; ++sweeps) {
        double off2 = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                if (i != j) off2 += creal(A[i * n + j] * conj(A[i * n + j]));
        if (off2 <= 1e-28 * fro2 || off2 == 0.0) { converged = 1; break; }
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                cplx z = A[p * n + q];
                double az = cabs(z);
                if (az == 0.0) continue;
                double app = creal(A[p * n + p]), aqq = creal(A[q * n + q]);
                double zeta = (aqq - app) / (2.0 * az);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = t * c;
                cplx w = z / az;
                /* A <- A U (columns p and q). */
                for (int k = 0; k < n; ++k) {
                    cplx akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * conj(w) * akq;
                    A[k * n + q] = s * w * akp + c * akq;
                }
                /* A <- U^H A (rows p and q). */
                for (int k = 0; k < n; ++k) {
                    cplx apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * w * aqk;
                    A[q * n + k] = s * conj(w) * apk + c * aqk;
                }
                A[p * n + q] = 0.0;
                A[q * n + p] = 0.0;
                A[p * n + p] = creal(A[p * n + p]);
                A[q * n + q] = creal(A[q * n + q]);
            }
        }
    }
    for (int i = 0; i < n; ++i) eig[i] = creal(A[i * n + i]);
    qsort(eig, (size_t)n, sizeof(double), cmp_double);
    return converged ? sweeps : -1;
}

/* Grand-canonical free energy of free fermions with one-particle energies
 * eig: F = -T sum_k ln(1 + exp(-(eps_k - mu)/T)), evaluated as
 * -T sum_k softplus(x_k), softplus(x) = max(x,0) + log1p(exp(-|x|)). */
double oracle_free_energy(int n, const double* eig, double mu, double T)
{
    double acc = 0.0;
    for (int k = 0; k < n; ++k) {
        double x = -(eig[k] - mu) / T;
        acc += (x > 0.0 ? x : 0.0) + log1p(exp(-fabs(x)));
    }
    return -T * acc;
}

/* Classical energy of the window of update site `site`: the sum over its
 * sites of (U/4)(m_i^2 - 1) (model 1) or K/2 x_i^2 - lambda x_i + mu
 * (model 2), the update site's variable replaced by s_new when given; zero
 * for model 0. */
static double window_classical(const oracle_model* m, const double* S, int site, const double* s_new)
{
    if (m->model != 1 && m->model != 2) return 0.0;
    window win = window_of(m, site);
    double acc = 0.0;
    for (int wz = 0; wz < win.ez; ++wz)
    for (int wy = 0; wy < win.ey; ++wy)
        for (int wx = 0; wx < win.ex; ++wx) {
            int g = window_site(m, &win, wx, wy, wz);
            const double* v = (s_new && g == site) ? s_new : S + 3 * g;
            if (m->model == 1)
                acc += 0.25 * m->U * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2] - 1.0);
            else
                acc += 0.5 * m->K * v[0] * v[0] - m->lam * v[0] + m->mu;
        }
    return acc;
}

/* Cluster free energy at update site `site` (spin replaced when s_new): the
 * one-body free energy of the cluster matrix plus, for model 1, the classical
 * energy of the window. */
static double cluster_F(const oracle_model* m, const double* S, int site, const double* s_new,
                        cplx* Hbuf, double* ebuf, int* n_out)
{
    int n = oracle_cluster_hamiltonian(m, S, site, s_new, Hbuf, NULL, NULL);
    oracle_eigvalsh_jacobi(n, Hbuf, ebuf);
    if (n_out) *n_out = n;
    return oracle_free_energy(n, ebuf, m->mu, m->T) + window_classical(m, S, site, s_new);
}

/* ------------------------------------------------------------------------ */
/* Schedules (Sec. III.a).  A schedule is an ordered list of stages; each    */
/* stage lists update sites.  Flattened, every site appears exactly once.    */
/*   tiled: stage (ax, ay, az) holds the sites (ax + s p, ay + s q, az + s r), */
/*          row-major; stages in row-major order of (ax, ay, az).             */
/*   block: the lattice is cut in two along each axis (2^d blocks, Sec.     */
/*          III.a: four blocks in two dimensions, eight in three); a stage   */
/*          is one block, its sites in row-major order; blocks row-major.     */
/* Writes stage_start[nstages+1] and sites[N]; returns nstages.               */
/* ------------------------------------------------------------------------ */
int oracle_schedule(const oracle_model* m, int32_t* stage_start, int32_t* sites)
{
    int Lx = m->Lx, Ly = m->Ly, Lz = m->Lz, ns = 0, pos = 0;
    stage_start[0] = 0;
    if (m->schedule == 0) {
        int s = m->stride;
        int sy = (Ly == 1) ? 1 : s, sz = (Lz == 1) ? 1 : s;
        for (int az = 0; az < sz && az < Lz; ++az)
            for (int ay = 0; ay < sy && ay < Ly; ++ay)
                for (int ax = 0; ax < s && ax < Lx; ++ax) {
                    for (int z = az; z < Lz; z += sz)
                        for (int y = ay; y < Ly; y += sy)
                            for (int x = ax; x < Lx; x += s) sites[pos++] = (z * Ly + y) * Lx + x;
                    stage_start[++ns] = pos;
                }
    } else {
        int hx = (Lx + 1) / 2, hy = (Ly + 1) / 2, hz = (Lz + 1) / 2;
        int nby = (Ly == 1) ? 1 : 2, nbz = (Lz == 1) ? 1 : 2;
        for (int bz = 0; bz < nbz; ++bz)
            for (int by = 0; by < nby; ++by)
                for (int bx = 0; bx < 2; ++bx) {
                    int xa = bx ? hx : 0, xb = bx ? Lx : hx;
                    int ya = (Ly == 1) ? 0 : (by ? hy : 0), yb = (Ly == 1) ? 1 : (by ? Ly : hy);
                    int za = (Lz == 1) ? 0 : (bz ? hz : 0), zb = (Lz == 1) ? 1 : (bz ? Lz : hz);
                    for (int z = za; z < zb; ++z)
                        for (int y = ya; y < yb; ++y)
                            for (int x = xa; x < xb; ++x) sites[pos++] = (z * Ly + y) * Lx + x;
                    if (pos > stage_start[ns]) stage_start[++ns] = pos;
                }
    }
    return ns;
}

/* Window membership: is lattice site g inside the window of update site c? */
int oracle_in_window(const oracle_model* m, int c, int g)
{
    window win = window_of(m, c);
    for (int wz = 0; wz < win.ez; ++wz)
        for (int wy = 0; wy < win.ey; ++wy)
            for (int wx = 0; wx < win.ex; ++wx)
                if (window_site(m, &win, wx, wy, wz) == g) return 1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One sequential TCA sweep (Sec. II.c, steps a-f), visiting the sites in the */
/* flattened stage order.  Each visit reads the current spins:                */
/*   a. gather the window;  b. build H_clus and diagonalise;                 */
/*   c. propose a new spin; d. rebuild with it and rediagonalise;            */
/*   e. Metropolis: accept iff ln u < -(F_new - F_old)/T;                    */
/*   f. on acceptance write the new spin.                                    */
/* Per visit (flattened order) the optional record arrays receive the site,  */
/* F_old, F_new, ln u and the decision.  Returns the number of acceptances,  */
/* or -1 on allocation failure.                                              */
/* ------------------------------------------------------------------------ */
int oracle_sweep(const oracle_model* m, double* S, uint64_t sweep,
                 int32_t* rec_site, double* rec_Fold, double* rec_Fnew,
                 double* rec_lnu, uint8_t* rec_acc)
{
    int N = n_sites(m);
    int nmax = n_max(m);
    int32_t* stage_start = malloc(sizeof(int32_t) * (size_t)(N + 1));
    int32_t* sites = malloc(sizeof(int32_t) * (size_t)N);
    cplx* H = malloc(sizeof(cplx) * (size_t)nmax * (size_t)nmax);
    double* e = malloc(sizeof(double) * (size_t)nmax);
    if (!stage_start || !sites || !H || !e) {
        free(stage_start); free(sites); free(H); free(e);
        return -1;
    }
    int ns = oracle_schedule(m, stage_start, sites);
    int nacc = 0;
    for (int st = 0; st < ns; ++st) {
        for (int k = stage_start[st]; k < stage_start[st + 1]; ++k) {
            int site = sites[k];
            double s_new[3];
            double F_old = cluster_F(m, S, site, NULL, H, e, NULL);
            oracle_propose(m, sweep, site, S + 3 * site, s_new);
            double F_new = cluster_F(m, S, site, s_new, H, e, NULL);
            double u[2];
            oracle_uniform2(m->seed, sweep, (uint32_t)site, PURPOSE_ACCEPT, u);
            double lnu = log(u[0]);
            int acc = lnu < -(F_new - F_old) / m->T;
            if (acc) {
                S[3 * site + 0] = s_new[0];
                S[3 * site + 1] = s_new[1];
                S[3 * site + 2] = s_new[2];
                ++nacc;
            }
            if (rec_site) rec_site[k] = site;
            if (rec_Fold) rec_Fold[k] = F_old;
            if (rec_Fnew) rec_Fnew[k] = F_new;
            if (rec_lnu) rec_lnu[k] = lnu;
            if (rec_acc) rec_acc[k] = (uint8_t)acc;
        }
    }
    free(stage_start); free(sites); free(H); free(e);
    return nacc;
}

/* Metropolis chain on a single site with every other spin frozen (used by
 * the distribution test of steps c-f).  Runs `steps` proposals at `site`
 * using sweep counters sweep0, sweep0+1, ...; writes the spin after each
 * step into trace (steps*3).  Returns the number of acceptances. */
int oracle_single_site_chain(const oracle_model* m, double* S, int site, uint64_t sweep0,
                             int steps, double* trace)
{
    int nmax = n_max(m);
    cplx* H = malloc(sizeof(cplx) * (size_t)nmax * (size_t)nmax);
    double* e = malloc(sizeof(double) * (size_t)nmax);
    if (!H || !e) { free(H); free(e); return -1; }
    int nacc = 0;
    double F_old = cluster_F(m, S, site, NULL, H, e, NULL);
    for (int k = 0; k < steps; ++k) {
        uint64_t sw = sweep0 + (uint64_t)k;
        double s_new[3], u[2];
        oracle_propose(m, sw, site, S + 3 * site, s_new);
        double F_new = cluster_F(m, S, site, s_new, H, e, NULL);
        oracle_uniform2(m->seed, sw, (uint32_t)site, PURPOSE_ACCEPT, u);
        if (log(u[0]) < -(F_new - F_old) / m->T) {
            memcpy(S + 3 * site, s_new, sizeof(s_new));
            F_old = F_new;
            ++nacc;
        }
        memcpy(trace + 3 * k, S + 3 * site, 3 * sizeof(double));
    }
    free(H); free(e);
    return nacc;
}

/* Cluster free energy of the current state at one site (for tests). */
double oracle_cluster_free_energy(const oracle_model* m, const double* S, int site, const double* s_new)
{
    int nmax = n_max(m);
    cplx* H = malloc(sizeof(cplx) * (size_t)nmax * (size_t)nmax);
    double* e = malloc(sizeof(double) * (size_t)nmax);
    double F = NAN;
    if (H && e) F = cluster_F(m, S, site, s_new, H, e, NULL);
    free(H); free(e);
    return F;
}

/* Magnetic structure factor of one configuration (Eq. 2 without the thermal
 * average): S(q) = (1/N^2) sum_{i,j} exp(i q.(r_i - r_j)) S_i . S_j, written
 * as the plain double sum over an Lx x Ly x Lz lattice. */
double oracle_structure_factor3(int Lx, int Ly, int Lz, const double* S, double qx, double qy, double qz)
{
    int N = Lx * Ly * Lz;
    double acc = 0.0;
    for (int i = 0; i < N; ++i) {
        double xi = i % Lx, yi = (i / Lx) % Ly, zi = i / (Lx * Ly);
        for (int j = 0; j < N; ++j) {
            double xj = j % Lx, yj = (j / Lx) % Ly, zj = j / (Lx * Ly);
            double dot = S[3 * i] * S[3 * j] + S[3 * i + 1] * S[3 * j + 1] + S[3 * i + 2] * S[3 * j + 2];
            acc += cos(qx * (xi - xj) + qy * (yi - yj) + qz * (zi - zj)) * dot;
        }
    }
    return acc / ((double)N * (double)N);
}

double oracle_structure_factor(int Lx, int Ly, const double* S, double qx, double qy)
{
    return oracle_structure_factor3(Lx, Ly, 1, S, qx, qy, 0.0);
}
