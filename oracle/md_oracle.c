/*
 * md_oracle.c - plain, slow FP64 CPU oracle for the short-range MD hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * constant with the CUDA library; it is compiled with -ffp-contract=off so
 * every expression below is evaluated exactly in the order written.
 *
 * What it computes (Meyer 2013, arXiv:1305.4196, and textbook MD):
 *   - the problem statement of Sec. I: N particles in a periodic box whose
 *     interactions vanish beyond a cutoff r_cut;
 *   - the linked-cell technique of Sec. II.A (cells at least as wide as the
 *     search radius, a particle interacts only with particles in its own or
 *     the 26 surrounding cells) - used here only to enumerate the pairs of
 *     the plain definition faster; a brute-force O(N^2) enumerator gives the
 *     same pair set bit for bit;
 *   - neighbour (Verlet) lists of Sec. II.A: all pairs closer than
 *     r_list = r_cut + skin at the build positions;
 *   - each pair counted once (Newton's third law, Sec. II.D.3);
 *   - Lennard-Jones pair energy u(r) = 4 eps [(s/r)^12 - (s/r)^6], force
 *     -du/dr along the pair vector, cut (unshifted) at r_cut;
 *   - per-pair virial W_ab = sum over pairs of d_a f_b;
 *   - velocity-Verlet integration (the paper only says "integration of the
 *     equations of motion", Sec. II.A) with a neighbour rebuild whenever some
 *     particle moved more than skin/2 since the last build (or every k steps,
 *     the paper's own protocol, Sec. III);
 *   - serial execution, as the paper's single-thread scheduler (Sec. II.C);
 *     one extra form, orc_lj_forces_full_omp / orc_run_nve_omp, sums each
 *     atom's full neighbour set on every host core (one writer per atom, the
 *     rule of Sec. II.A) for the timed CPU baseline, pinned against the serial
 *     definition by the CPU tests;
 *   - the same velocity-Verlet loop around the many-body TB-SMA forces
 *     (orc_run_nve_tbsma, Sec. III's potential).
 *
 * Readings where the paper is silent (potential, integrator, rebuild rule,
 * strict '<' at both cutoffs, minimum image by rint) are the ones listed in
 * the repository's design notes.  All parity of this file is pinned by the
 * CPU tests (closed forms, finite differences, brute force, lattice sums).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- helpers */

/* Minimum-image displacement component: d - L * rint(d / L). */
static double mic(double d, double L)
{
    return d - L * nearbyint(d / L);
}

/* x_i - x_j under minimum image; returns |d|^2 summed in x, y, z order. */
static double pair_disp(const double *x, int64_t i, int64_t j, const double *box, double d[3])
{
    d[0] = mic(x[3 * i + 0] - x[3 * j + 0], box[0]);
    d[1] = mic(x[3 * i + 1] - x[3 * j + 1], box[1]);
    d[2] = mic(x[3 * i + 2] - x[3 * j + 2], box[2]);
    return d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
}

typedef void (*pair_fn)(void *ctx, int64_t i, int64_t j, const double d[3], double r2);

/*
 * Call fn(i, j, d, r2) once for every unordered pair i < j with r2 < r*r.
 * brute != 0 forces the O(N^2) loop; otherwise linked cells of width >= r
 * are used when every dimension holds at least 3 of them.
 */
static void for_each_pair(int64_t n, const double *x, const double *box, double r,
                          int brute, pair_fn fn, void *ctx)
{
    const double r2max = r * r;
    int nc[3];
    for (int k = 0; k < 3; ++k) {
        nc[k] = (int)floor(box[k] / r);
        if (nc[k] < 1) nc[k] = 1;
    }
    if (brute || nc[0] < 3 || nc[1] < 3 || nc[2] < 3) {
        double d[3];
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = i + 1; j < n; ++j) {
                double r2 = pair_disp(x, i, j, box, d);
                if (r2 < r2max) fn(ctx, i, j, d, r2);
            }
        return;
    }
    /* linked cells: head[c] is the first particle of cell c, next[i] the one after i */
    const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * ncell);
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    int32_t *cell = (int32_t *)malloc(sizeof(int32_t) * 3 * (n > 0 ? n : 1));
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    for (int64_t i = n - 1; i >= 0; --i) {
        int cc[3];
        for (int k = 0; k < 3; ++k) {
            double w = box[k] / nc[k];
            double xk = x[3 * i + k] - box[k] * floor(x[3 * i + k] / box[k]);
            int c = (int)floor(xk / w);
            if (c < 0) c = 0;
            if (c >= nc[k]) c = nc[k] - 1;
            cc[k] = c;
            cell[3 * i + k] = c;
        }
        int64_t c = ((int64_t)cc[2] * nc[1] + cc[1]) * nc[0] + cc[0];
        next[i] = head[c];
        head[c] = i;
    }
    double d[3];
    for (int64_t i = 0; i < n; ++i) {
        for (int oz = -1; oz <= 1; ++oz)
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    int cx = (cell[3 * i + 0] + ox + nc[0]) % nc[0];
                    int cy = (cell[3 * i + 1] + oy + nc[1]) % nc[1];
                    int cz = (cell[3 * i + 2] + oz + nc[2]) % nc[2];
                    int64_t c = ((int64_t)cz * nc[1] + cy) * nc[0] + cx;
                    for (int64_t j = head[c]; j >= 0; j = next[j]) {
                        if (j <= i) continue;
                        double r2 = pair_disp(x, i, j, box, d);
                        if (r2 < r2max) fn(ctx, i, j, d, r2);
                    }
                }
    }
    free(head);
    free(next);
    free(cell);
}

/* ------------------------------------------------------- neighbour pairs */

typedef struct {
    int64_t count, cap;
    int32_t *pairs; /* nullable: 2 x cap */
} pair_sink;

static void collect_pair(void *ctx, int64_t i, int64_t j, const double d[3], double r2)
{
    (void)d;
    (void)r2;
    pair_sink *s = (pair_sink *)ctx;
    if (s->pairs && s->count < s->cap) {
        s->pairs[2 * s->count + 0] = (int32_t)i;
        s->pairs[2 * s->count + 1] = (int32_t)j;
    }
    s->count++;
}

static int cmp_pair(const void *a, const void *b)
{
    const int32_t *p = (const int32_t *)a, *q = (const int32_t *)b;
    if (p[0] != q[0]) return p[0] < q[0] ? -1 : 1;
    if (p[1] != q[1]) return p[1] < q[1] ? -1 : 1;
    return 0;
}

/*
 * Neighbour set at positions x: all pairs (i, j), i < j, with minimum-image
 * |x_i - x_j|^2 < r_list^2 (strict).  Returns the number of pairs; if pairs is
 * non-null and cap is large enough they are written sorted by (i, j).
 */
int64_t orc_neighbor_pairs(int64_t n, const double *x, const double *box, double r_list,
                           int brute, int64_t cap, int32_t *pairs)
{
    pair_sink s = {0, cap, pairs};
    for_each_pair(n, x, box, r_list, brute, collect_pair, &s);
    if (pairs && s.count <= cap) qsort(pairs, (size_t)s.count, 2 * sizeof(int32_t), cmp_pair);
    return s.count;
}

/* ------------------------------------------------------- Lennard-Jones */

/* Neumaier compensated sum: keeps the rounding error of a long sum of pair
 * terms near one ulp of the result, so whole-system totals are accurate far
 * below the 1e-12 relative parity bar at any system size. */
typedef struct {
    double s, c;
} csum;

static void csum_add(csum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double csum_get(const csum *a) { return a->s + a->c; }

typedef struct {
    int32_t nsp;
    const double *eps, *sig, *rc; /* nsp x nsp, row-major, symmetric */
    const int32_t *species;       /* nullable: all species 0 */
    double *f;                    /* N x 3, accumulated */
    double *pe_atom;              /* nullable: N, half of each pair energy */
    csum pe, vir[6];
} lj_acc;

/* One pair: energy, force on i (= -force on j) and virial, if r < r_cut(a,b). */
static void lj_pair(void *ctx, int64_t i, int64_t j, const double d[3], double r2)
{
    lj_acc *a = (lj_acc *)ctx;
    int32_t si = a->species ? a->species[i] : 0;
    int32_t sj = a->species ? a->species[j] : 0;
    int32_t t = si * a->nsp + sj;
    double rc = a->rc[t];
    if (!(r2 < rc * rc)) return;
    double s = a->sig[t];
    double e = a->eps[t];
    double sr2 = (s * s) / r2;
    double s6 = sr2 * sr2 * sr2;
    double u = 4.0 * e * (s6 * s6 - s6);
    double fr = 24.0 * e * (2.0 * s6 * s6 - s6) / r2; /* |f| / r, positive = repulsive */
    for (int k = 0; k < 3; ++k) {
        a->f[3 * i + k] += fr * d[k];
        a->f[3 * j + k] -= fr * d[k];
    }
    csum_add(&a->pe, u);
    if (a->pe_atom) {
        a->pe_atom[i] += 0.5 * u;
        a->pe_atom[j] += 0.5 * u;
    }
    csum_add(&a->vir[0], d[0] * (fr * d[0]));
    csum_add(&a->vir[1], d[1] * (fr * d[1]));
    csum_add(&a->vir[2], d[2] * (fr * d[2]));
    csum_add(&a->vir[3], d[0] * (fr * d[1]));
    csum_add(&a->vir[4], d[0] * (fr * d[2]));
    csum_add(&a->vir[5], d[1] * (fr * d[2]));
}

static double max_cut(int32_t nsp, const double *rc)
{
    double m = 0.0;
    for (int32_t t = 0; t < nsp * nsp; ++t)
        if (rc[t] > m) m = rc[t];
    return m;
}

/*
 * Forces, total potential energy and virial of the whole system at x: the
 * plain definition, every pair closer than its cutoff counted once.
 * f (N x 3) is overwritten; pe_atom (nullable) receives half of each pair energy.
 */
void orc_lj_forces(int64_t n, const double *x, const double *box, const int32_t *species,
                   int32_t nsp, const double *eps, const double *sig, const double *rc,
                   int brute, double *f, double *pe_atom, double *pe, double *vir)
{
    memset(f, 0, sizeof(double) * 3 * (size_t)n);
    if (pe_atom) memset(pe_atom, 0, sizeof(double) * (size_t)n);
    lj_acc a;
    memset(&a, 0, sizeof(a));
    a.nsp = nsp;
    a.eps = eps;
    a.sig = sig;
    a.rc = rc;
    a.species = species;
    a.f = f;
    a.pe_atom = pe_atom;
    for_each_pair(n, x, box, max_cut(nsp, rc), brute, lj_pair, &a);
    if (pe) *pe = csum_get(&a.pe);
    if (vir)
        for (int k = 0; k < 6; ++k) vir[k] = csum_get(&a.vir[k]);
}

/*
 * Forces restricted to a given pair set (each unordered pair once), as a
 * neighbour list is used between rebuilds: only listed pairs closer than
 * their cutoff contribute.
 */
void orc_lj_forces_pairs(int64_t n, const double *x, const double *box, const int32_t *species,
                         int32_t nsp, const double *eps, const double *sig, const double *rc,
                         int64_t npairs, const int32_t *pairs, double *f, double *pe, double *vir)
{
    memset(f, 0, sizeof(double) * 3 * (size_t)n);
    lj_acc a;
    memset(&a, 0, sizeof(a));
    a.nsp = nsp;
    a.eps = eps;
    a.sig = sig;
    a.rc = rc;
    a.species = species;
    a.f = f;
    double d[3];
    for (int64_t p = 0; p < npairs; ++p) {
        int64_t i = pairs[2 * p], j = pairs[2 * p + 1];
        double r2 = pair_disp(x, i, j, box, d);
        lj_pair(&a, i, j, d, r2);
    }
    if (pe) *pe = csum_get(&a.pe);
    if (vir)
        for (int k = 0; k < 6; ++k) vir[k] = csum_get(&a.vir[k]);
}

/*
 * Force, energy share and virial share on each of m sampled atoms, by a
 * direct loop over all N partners (O(m N)).  Used to check single atoms of
 * systems too large for a whole-system oracle run.  vir_out is m x 6.
 */
void orc_lj_forces_subset(int64_t n, const double *x, const double *box, const int32_t *species,
                          int32_t nsp, const double *eps, const double *sig, const double *rc,
                          int64_t m, const int64_t *idx, double *f_out, double *pe_out, double *vir_out)
{
    double d[3];
    for (int64_t q = 0; q < m; ++q) {
        int64_t i = idx[q];
        int32_t si = species ? species[i] : 0;
        double f[3] = {0.0, 0.0, 0.0}, pe = 0.0, w[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            int32_t sj = species ? species[j] : 0;
            int32_t t = si * nsp + sj;
            double r2 = pair_disp(x, i, j, box, d);
            double rcut = rc[t];
            if (!(r2 < rcut * rcut)) continue;
            double s = sig[t], e = eps[t];
            double sr2 = (s * s) / r2;
            double s6 = sr2 * sr2 * sr2;
            double u = 4.0 * e * (s6 * s6 - s6);
            double fr = 24.0 * e * (2.0 * s6 * s6 - s6) / r2;
            for (int k = 0; k < 3; ++k) f[k] += fr * d[k];
            pe += 0.5 * u;
            w[0] += 0.5 * (d[0] * (fr * d[0]));
            w[1] += 0.5 * (d[1] * (fr * d[1]));
            w[2] += 0.5 * (d[2] * (fr * d[2]));
            w[3] += 0.5 * (d[0] * (fr * d[1]));
            w[4] += 0.5 * (d[0] * (fr * d[2]));
            w[5] += 0.5 * (d[1] * (fr * d[2]));
        }
        for (int k = 0; k < 3; ++k) f_out[3 * q + k] = f[k];
        if (pe_out) pe_out[q] = pe;
        if (vir_out)
            for (int k = 0; k < 6; ++k) vir_out[6 * q + k] = w[k];
    }
}

/* ------------------------------------------------------- gradients */

/*
 * Reverse-mode derivatives of the Lennard-Jones forces, for force matching.
 * L is any scalar function of the forces; G = dL/dF is given (N x 3).  With
 * f_ij = g(r^2) d the force of pair (i,j) on i (d = x_i - x_j), the chain rule
 * over the pairs closer than their cutoff (the pair set held fixed: the cutoff
 * itself contributes no derivative) gives, with w = G_i - G_j:
 *   dL/dx_i += g w + 2 g' (w . d) d,   dL/dx_j -= the same      (Hessian-vector product)
 *   dL/deps_ab += (w . d) g / eps
 *   dL/dsig_ab += (w . d) dg/dsig,  dg/dsig = 144 eps (4 s6^2 - s6) / (sig r^2)
 * where g = 24 eps (2 s6^2 - s6) / r^2, s6 = (sig^2 / r^2)^3 and
 * g' = dg/d(r^2) = 24 eps (4 s6 - 14 s6^2) / r^4.
 * The species tables are symmetric: the derivative with respect to the shared value
 * of an unordered species pair {a,b} is written to both [a][b] and [b][a].
 * Also the energy's parameter derivatives dE/deps_ab = sum u / eps and
 * dE/dsig_ab = sum 24 eps (2 s6^2 - s6) / sig (nullable outputs).
 */
typedef struct {
    int32_t nsp;
    const double *eps, *sig, *rc;
    const int32_t *species;
    const double *G;
    double *gx;
    csum *geps, *gsig, *eeps, *esig; /* per unordered species pair, index a * nsp + b with a <= b */
    int absmode;                     /* sum |term| instead of term for geps, gsig (a sum's scale) */
} lj_grad_acc;

static void lj_grad_pair(void *ctx, int64_t i, int64_t j, const double d[3], double r2)
{
    lj_grad_acc *a = (lj_grad_acc *)ctx;
    int32_t si = a->species ? a->species[i] : 0;
    int32_t sj = a->species ? a->species[j] : 0;
    int32_t t = si * a->nsp + sj;
    double rc = a->rc[t];
    if (!(r2 < rc * rc)) return;
    int32_t u = si <= sj ? si * a->nsp + sj : sj * a->nsp + si;
    double s = a->sig[t];
    double e = a->eps[t];
    double sr2 = (s * s) / r2;
    double s6 = sr2 * sr2 * sr2;
    double g = 24.0 * e * (2.0 * s6 * s6 - s6) / r2;
    if (a->G) {
        double w[3], wd = 0.0;
        for (int k = 0; k < 3; ++k) {
            w[k] = a->G[3 * i + k] - a->G[3 * j + k];
            wd += w[k] * d[k];
        }
        double gp = 24.0 * e * (4.0 * s6 - 14.0 * s6 * s6) / (r2 * r2);
        for (int k = 0; k < 3; ++k) {
            double h = g * w[k] + 2.0 * gp * wd * d[k];
            a->gx[3 * i + k] += h;
            a->gx[3 * j + k] -= h;
        }
        double te = wd * (g / e);
        double ts = wd * (144.0 * e * (4.0 * s6 * s6 - s6) / (s * r2));
        csum_add(&a->geps[u], a->absmode ? fabs(te) : te);
        csum_add(&a->gsig[u], a->absmode ? fabs(ts) : ts);
    }
    if (a->eeps) {
        csum_add(&a->eeps[u], 4.0 * (s6 * s6 - s6));
        csum_add(&a->esig[u], 24.0 * e * (2.0 * s6 * s6 - s6) / s);
    }
}

static void lj_grad_run(int64_t n, const double *x, const double *box, const int32_t *species, int32_t nsp,
                        const double *eps, const double *sig, const double *rc, const double *G, double *gx,
                        double *geps, double *gsig, double *dE_deps, double *dE_dsig, int absmode)
{
    csum acc[4][64];
    memset(acc, 0, sizeof(acc));
    lj_grad_acc a;
    memset(&a, 0, sizeof(a));
    a.absmode = absmode;
    a.nsp = nsp;
    a.eps = eps;
    a.sig = sig;
    a.rc = rc;
    a.species = species;
    a.G = G;
    a.gx = gx;
    a.geps = acc[0];
    a.gsig = acc[1];
    if (dE_deps) {
        a.eeps = acc[2];
        a.esig = acc[3];
    }
    if (G) memset(gx, 0, sizeof(double) * 3 * (size_t)n);
    for_each_pair(n, x, box, max_cut(nsp, rc), 0, lj_grad_pair, &a);
    for (int32_t p = 0; p < nsp; ++p)
        for (int32_t q = 0; q < nsp; ++q) {
            int32_t u = p <= q ? p * nsp + q : q * nsp + p;
            if (G) {
                geps[p * nsp + q] = csum_get(&acc[0][u]);
                gsig[p * nsp + q] = csum_get(&acc[1][u]);
            }
            if (dE_deps) {
                dE_deps[p * nsp + q] = csum_get(&acc[2][u]);
                dE_dsig[p * nsp + q] = csum_get(&acc[3][u]);
            }
        }
}

void orc_lj_grad(int64_t n, const double *x, const double *box, const int32_t *species, int32_t nsp,
                 const double *eps, const double *sig, const double *rc, const double *G, double *gx,
                 double *geps, double *gsig, double *dE_deps, double *dE_dsig)
{
    lj_grad_run(n, x, box, species, nsp, eps, sig, rc, G, gx, geps, gsig, dE_deps, dE_dsig, 0);
}

/*
 * The scale of the parameter sums of orc_lj_grad: sum over the pairs of |term| for
 * dL/deps_ab and dL/dsig_ab (same tables).  A sum whose terms each carry a relative
 * error e is off by at most e times this scale, however much its terms cancel.
 */
void orc_lj_grad_abs(int64_t n, const double *x, const double *box, const int32_t *species, int32_t nsp,
                     const double *eps, const double *sig, const double *rc, const double *G, double *gx_scratch,
                     double *geps_abs, double *gsig_abs)
{
    lj_grad_run(n, x, box, species, nsp, eps, sig, rc, G, gx_scratch, geps_abs, gsig_abs, NULL, NULL, 1);
}

/* ------------------------------------------------------- many-body (TB-SMA) */

/*
 * The tight-binding second-moment potential of Cleri and Rosato (Phys. Rev. B 48,
 * 22 (1993)), the potential of all of the paper's benchmarks (Sec. III):
 *   E = sum_i [ sum_j phi(r_ij) - sqrt(rho_i) ],  rho_i = sum_j psi(r_ij),
 *   phi(r) = A exp(-p (r / r0 - 1)),  psi(r) = xi^2 exp(-2 q (r / r0 - 1)),
 * both sums over the neighbours j of i closer than r_cut (strict <).  The force on i,
 * -dE/dx_i, is a sum over the same pairs with d = x_i - x_j:
 *   F_i = sum_j [ (2 p / r0) phi - (q / r0) psi (1 / sqrt(rho_i) + 1 / sqrt(rho_j)) ] d / r
 * (the repulsion of a pair enters E twice, once per atom; the band term of atom k
 * depends on every neighbour's distance).  An atom with no neighbour has rho = 0 and
 * no force.  Two passes in the definition's order: the densities, then the forces.
 * Per-atom energy: sum_j phi - sqrt(rho_i); the virial is sum over pairs of d_a f_b.
 * prm = {A, xi, p, q, r0}.
 */
typedef struct {
    const double *prm;
    double rc;
    double *rho;       /* N, accumulated */
    csum *rho_acc;     /* N compensated sums */
    csum rep;
    double *f;
    const double *inv; /* N: 1 / sqrt(rho), 0 without neighbours */
    double *e_atom;    /* nullable */
    csum vir[6];
} tb_acc;

static void tb_density_pair(void *ctx, int64_t i, int64_t j, const double d[3], double r2)
{
    tb_acc *a = (tb_acc *)ctx;
    (void)d;
    if (!(r2 < a->rc * a->rc)) return;
    const double A = a->prm[0], xi = a->prm[1], p = a->prm[2], q = a->prm[3], r0 = a->prm[4];
    double r = sqrt(r2);
    double psi = xi * xi * exp(-2.0 * q * (r / r0 - 1.0));
    double phi = A * exp(-p * (r / r0 - 1.0));
    csum_add(&a->rho_acc[i], psi);
    csum_add(&a->rho_acc[j], psi);
    csum_add(&a->rep, 2.0 * phi);
    if (a->e_atom) {
        a->e_atom[i] += phi;
        a->e_atom[j] += phi;
    }
}

static void tb_force_pair(void *ctx, int64_t i, int64_t j, const double d[3], double r2)
{
    tb_acc *a = (tb_acc *)ctx;
    if (!(r2 < a->rc * a->rc)) return;
    const double A = a->prm[0], xi = a->prm[1], p = a->prm[2], q = a->prm[3], r0 = a->prm[4];
    double r = sqrt(r2);
    double psi = xi * xi * exp(-2.0 * q * (r / r0 - 1.0));
    double phi = A * exp(-p * (r / r0 - 1.0));
    double fr = (2.0 * p / r0) * phi - (q / r0) * psi * (a->inv[i] + a->inv[j]); /* along d / r */
    double g = fr / r;
    for (int k = 0; k < 3; ++k) {
        a->f[3 * i + k] += g * d[k];
        a->f[3 * j + k] -= g * d[k];
    }
    csum_add(&a->vir[0], d[0] * (g * d[0]));
    csum_add(&a->vir[1], d[1] * (g * d[1]));
    csum_add(&a->vir[2], d[2] * (g * d[2]));
    csum_add(&a->vir[3], d[0] * (g * d[1]));
    csum_add(&a->vir[4], d[0] * (g * d[2]));
    csum_add(&a->vir[5], d[1] * (g * d[2]));
}

/*
 * Forces (N x 3, overwritten), densities rho (nullable, N), per-atom energies
 * (nullable, N), total energy and virial (nullable) at x.
 */
void orc_tbsma_forces(int64_t n, const double *x, const double *box, const double *prm, double rc, int brute,
                      double *f, double *rho_out, double *e_atom, double *energy, double *vir)
{
    tb_acc a;
    memset(&a, 0, sizeof(a));
    a.prm = prm;
    a.rc = rc;
    a.rho_acc = (csum *)calloc((size_t)(n > 0 ? n : 1), sizeof(csum));
    double *inv = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    a.e_atom = e_atom;
    if (e_atom) memset(e_atom, 0, sizeof(double) * (size_t)n);
    for_each_pair(n, x, box, rc, brute, tb_density_pair, &a);
    csum band;
    memset(&band, 0, sizeof(band));
    for (int64_t i = 0; i < n; ++i) {
        double rho = csum_get(&a.rho_acc[i]);
        double sq = sqrt(rho);
        inv[i] = rho > 0.0 ? 1.0 / sq : 0.0;
        csum_add(&band, -sq);
        if (rho_out) rho_out[i] = rho;
        if (e_atom) e_atom[i] -= sq;
    }
    memset(f, 0, sizeof(double) * 3 * (size_t)n);
    a.f = f;
    a.inv = inv;
    for_each_pair(n, x, box, rc, brute, tb_force_pair, &a);
    if (energy) *energy = csum_get(&a.rep) + csum_get(&band);
    if (vir)
        for (int k = 0; k < 6; ++k) vir[k] = csum_get(&a.vir[k]);
    free(a.rho_acc);
    free(inv);
}

/* ------------------------------------------------------- integration */

/* Kinetic energy 1/2 sum m v^2 (mass per species). */
double orc_kinetic(int64_t n, const double *v, const int32_t *species, const double *mass)
{
    csum ke = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) {
        double m = mass[species ? species[i] : 0];
        csum_add(&ke, 0.5 * m * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]));
    }
    return csum_get(&ke);
}

/*
 * Velocity-Verlet run of nsteps with neighbour rebuilds, for any force field
 * (force(ctx, n, x, box, f, pe) overwrites f and the potential energy *pe).
 *
 * Per step: v += (dt/2m) F;  x += dt v;  rebuild test;  F = F(x);
 * v += (dt/2m) F.  The rebuild test (policy 0) fires when some particle's
 * squared displacement since the last build exceeds (skin/2)^2; policy 1
 * fires every k-th step.  A rebuild maps positions back into [0, L) (one
 * box length at most, counted in the image array) and records them as the
 * new reference positions.  Forces are the plain definition at every step.
 *
 * x, v, image (N x 3) are updated in place.  f_io (nullable, N x 3): with
 * f_given != 0 it holds the forces at the starting x and the run uses them
 * instead of evaluating them once more; on return it holds the forces at the
 * final x.  Optional per-step outputs (length nsteps): pe_hist, ke_hist.
 * Returns the number of rebuilds.
 */
typedef void (*force_eval_fn)(void *ctx, int64_t n, const double *x, const double *box, double *f, double *pe);

static int64_t vv_run(int64_t n, double *x, double *v, int32_t *image, const double *box,
                      const int32_t *species, int32_t nsp, const double *mass, double dt, double skin,
                      int32_t policy, int32_t every_k, int64_t nsteps, force_eval_fn force, void *fctx,
                      double *f_io, int32_t f_given, double *pe_hist, double *ke_hist)
{
    double *f = f_io ? f_io : (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *xref = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *hdtm = (double *)malloc(sizeof(double) * (size_t)nsp);
    for (int32_t s = 0; s < nsp; ++s) hdtm[s] = (0.5 * dt) / mass[s];
    memcpy(xref, x, sizeof(double) * 3 * (size_t)n);
    const double half_skin = 0.5 * skin;
    const double lim2 = half_skin * half_skin;
    double pe = 0.0;
    int64_t rebuilds = 0;
    if (!(f_io && f_given)) force(fctx, n, x, box, f, &pe);
    for (int64_t step = 0; step < nsteps; ++step) {
        for (int64_t i = 0; i < n; ++i) {
            double h = hdtm[species ? species[i] : 0];
            for (int k = 0; k < 3; ++k) {
                v[3 * i + k] = v[3 * i + k] + h * f[3 * i + k];
                x[3 * i + k] = x[3 * i + k] + dt * v[3 * i + k];
            }
        }
        int rebuild = 0;
        if (policy == 1) {
            rebuild = every_k > 0 && ((step + 1) % every_k) == 0;
        } else {
            for (int64_t i = 0; i < n && !rebuild; ++i) {
                double dx = x[3 * i] - xref[3 * i];
                double dy = x[3 * i + 1] - xref[3 * i + 1];
                double dz = x[3 * i + 2] - xref[3 * i + 2];
                if (dx * dx + dy * dy + dz * dz > lim2) rebuild = 1;
            }
        }
        if (rebuild) {
            for (int64_t i = 0; i < n; ++i)
                for (int k = 0; k < 3; ++k) {
                    double L = box[k];
                    if (x[3 * i + k] >= L) {
                        x[3 * i + k] -= L;
                        image[3 * i + k] += 1;
                    } else if (x[3 * i + k] < 0.0) {
                        x[3 * i + k] += L;
                        image[3 * i + k] -= 1;
                    }
                }
            memcpy(xref, x, sizeof(double) * 3 * (size_t)n);
            rebuilds++;
        }
        force(fctx, n, x, box, f, &pe);
        for (int64_t i = 0; i < n; ++i) {
            double h = hdtm[species ? species[i] : 0];
            for (int k = 0; k < 3; ++k) v[3 * i + k] = v[3 * i + k] + h * f[3 * i + k];
        }
        if (pe_hist) pe_hist[step] = pe;
        if (ke_hist) ke_hist[step] = orc_kinetic(n, v, species, mass);
    }
    if (!f_io) free(f);
    free(xref);
    free(hdtm);
    return rebuilds;
}

/* The Lennard-Jones model of orc_lj_forces as a force field of vv_run. */
typedef struct {
    const int32_t *species;
    int32_t nsp;
    const double *eps, *sig, *rc;
} lj_model;

static void lj_eval(void *ctx, int64_t n, const double *x, const double *box, double *f, double *pe)
{
    const lj_model *m = (const lj_model *)ctx;
    double vir[6];
    orc_lj_forces(n, x, box, m->species, m->nsp, m->eps, m->sig, m->rc, 0, f, NULL, pe, vir);
}

/* Velocity Verlet with the Lennard-Jones forces of orc_lj_forces (see vv_run). */
int64_t orc_run_nve(int64_t n, double *x, double *v, int32_t *image, const double *box,
                    const int32_t *species, int32_t nsp, const double *eps, const double *sig,
                    const double *rc, const double *mass, double dt, double skin,
                    int32_t policy, int32_t every_k, int64_t nsteps, double *f_io, int32_t f_given,
                    double *pe_hist, double *ke_hist)
{
    lj_model m = {species, nsp, eps, sig, rc};
    return vv_run(n, x, v, image, box, species, nsp, mass, dt, skin, policy, every_k, nsteps, lj_eval, &m,
                  f_io, f_given, pe_hist, ke_hist);
}

/* The many-body model of orc_tbsma_forces as a force field of vv_run. */
typedef struct {
    const double *prm;
    double rc;
} tb_model;

static void tb_eval(void *ctx, int64_t n, const double *x, const double *box, double *f, double *pe)
{
    const tb_model *m = (const tb_model *)ctx;
    orc_tbsma_forces(n, x, box, m->prm, m->rc, 0, f, NULL, NULL, pe, NULL);
}

/* Velocity Verlet with the TB-SMA forces of orc_tbsma_forces, one species of mass `mass`. */
int64_t orc_run_nve_tbsma(int64_t n, double *x, double *v, int32_t *image, const double *box,
                          const double *prm, double rc, double mass, double dt, double skin,
                          int32_t policy, int32_t every_k, int64_t nsteps, double *pe_hist, double *ke_hist)
{
    tb_model m = {prm, rc};
    return vv_run(n, x, v, image, box, NULL, 1, &mass, dt, skin, policy, every_k, nsteps, tb_eval, &m,
                  NULL, 0, pe_hist, ke_hist);
}

/* ------------------------------------------------------- all host cores */

/*
 * Lennard-Jones forces by full neighbour sums on every host core: the force on
 * atom i is the sum over all j != i closer than their cutoff of the pair
 * force f_ij, each atom summed by one thread that writes only that atom (the
 * full-list form of the paper's cell tasks, Sec. II.A: no particle is written
 * by two threads, so no locks or reductions are needed).  Each pair is thus
 * evaluated twice, once from each side; the result equals orc_lj_forces up to
 * the order of the additions.  Linked cells of width >= the largest cutoff
 * when every dimension holds at least 3, else all pairs.  *pe is the total
 * potential energy (half of each pair per atom, summed in atom order).
 * Returns the number of threads used.
 */
int32_t orc_lj_forces_full_omp(int64_t n, const double *x, const double *box, const int32_t *species,
                               int32_t nsp, const double *eps, const double *sig, const double *rc,
                               double *f, double *pe)
{
    const double r = max_cut(nsp, rc);
    int nc[3];
    for (int k = 0; k < 3; ++k) {
        nc[k] = (int)floor(box[k] / r);
        if (nc[k] < 1) nc[k] = 1;
    }
    const int cells = nc[0] >= 3 && nc[1] >= 3 && nc[2] >= 3;
    const int64_t ncell = cells ? (int64_t)nc[0] * nc[1] * nc[2] : 1;
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * ncell);
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    int32_t *cell = (int32_t *)malloc(sizeof(int32_t) * 3 * (n > 0 ? n : 1));
    double *pe_atom = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    for (int64_t i = n - 1; i >= 0; --i) {
        int cc[3] = {0, 0, 0};
        if (cells)
            for (int k = 0; k < 3; ++k) {
                double w = box[k] / nc[k];
                double xk = x[3 * i + k] - box[k] * floor(x[3 * i + k] / box[k]);
                int c = (int)floor(xk / w);
                if (c < 0) c = 0;
                if (c >= nc[k]) c = nc[k] - 1;
                cc[k] = c;
            }
        for (int k = 0; k < 3; ++k) cell[3 * i + k] = cc[k];
        int64_t c = ((int64_t)cc[2] * nc[1] + cc[1]) * nc[0] + cc[0];
        if (!cells) c = 0;
        next[i] = head[c];
        head[c] = i;
    }
    int32_t threads = 1;
#pragma omp parallel
    {
#ifdef _OPENMP
#pragma omp single
        threads = (int32_t)omp_get_num_threads();
#endif
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) {
            double fi[3] = {0.0, 0.0, 0.0}, ui = 0.0, d[3];
            const int32_t si = species ? species[i] : 0;
            const int span = cells ? 1 : 0;
            for (int oz = -span; oz <= span; ++oz)
                for (int oy = -span; oy <= span; ++oy)
                    for (int ox = -span; ox <= span; ++ox) {
                        int64_t c = 0;
                        if (cells) {
                            int cx = (cell[3 * i + 0] + ox + nc[0]) % nc[0];
                            int cy = (cell[3 * i + 1] + oy + nc[1]) % nc[1];
                            int cz = (cell[3 * i + 2] + oz + nc[2]) % nc[2];
                            c = ((int64_t)cz * nc[1] + cy) * nc[0] + cx;
                        }
                        for (int64_t j = head[c]; j >= 0; j = next[j]) {
                            if (j == i) continue;
                            double r2 = pair_disp(x, i, j, box, d);
                            int32_t t = si * nsp + (species ? species[j] : 0);
                            if (!(r2 < rc[t] * rc[t])) continue;
                            double sr2 = (sig[t] * sig[t]) / r2;
                            double s6 = sr2 * sr2 * sr2;
                            double fr = 24.0 * eps[t] * (2.0 * s6 * s6 - s6) / r2;
                            for (int k = 0; k < 3; ++k) fi[k] += fr * d[k];
                            ui += 0.5 * (4.0 * eps[t] * (s6 * s6 - s6));
                        }
                    }
            for (int k = 0; k < 3; ++k) f[3 * i + k] = fi[k];
            pe_atom[i] = ui;
        }
    }
    if (pe) {
        csum acc = {0.0, 0.0};
        for (int64_t i = 0; i < n; ++i) csum_add(&acc, pe_atom[i]);
        *pe = csum_get(&acc);
    }
    free(head);
    free(next);
    free(cell);
    free(pe_atom);
    return threads;
}

static void lj_eval_omp(void *ctx, int64_t n, const double *x, const double *box, double *f, double *pe)
{
    const lj_model *m = (const lj_model *)ctx;
    orc_lj_forces_full_omp(n, x, box, m->species, m->nsp, m->eps, m->sig, m->rc, f, pe);
}

/* Velocity Verlet with the all-cores full-sum forces of orc_lj_forces_full_omp (see vv_run). */
int64_t orc_run_nve_omp(int64_t n, double *x, double *v, int32_t *image, const double *box,
                        const int32_t *species, int32_t nsp, const double *eps, const double *sig,
                        const double *rc, const double *mass, double dt, double skin,
                        int32_t policy, int32_t every_k, int64_t nsteps, double *f_io, int32_t f_given,
                        double *pe_hist, double *ke_hist)
{
    lj_model m = {species, nsp, eps, sig, rc};
    return vv_run(n, x, v, image, box, species, nsp, mass, dt, skin, policy, every_k, nsteps, lj_eval_omp, &m,
                  f_io, f_given, pe_hist, ke_hist);
}

/* Threads an OpenMP region of this library uses (1 when built without OpenMP). */
int32_t orc_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}
