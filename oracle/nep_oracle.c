/*
 * nep_oracle.c -- plain FP64 CPU oracle of the neuroevolution-potential (NEP)
 * hot path, written from the paper (Fan et al., arXiv 2107.08119).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant with
 * the CUDA library; both are written independently from the paper.
 *
 * Everything is double precision, evaluated literally in the order the paper
 * states it: the angular descriptor is the O(M^2) double sum over neighbour
 * pairs of Eq. 13 (not the spherical-harmonic rewrite), and the partial forces
 * are the explicit expressions of Eqs. 24-25.  Readings of points the paper
 * leaves open:
 *   - q_nl includes the k = j term of its double sum (Eq. 13 sums j != i and
 *     k != i only; Eq. 25's factor 2 and the addition-theorem link of
 *     Eqs. 17-18 both assume the diagonal term is present);
 *   - the radial functions inside q_nl use the angular cutoff r_c^A;
 *   - no descriptor normalisation; single species (no Z weighting, Eq. 19);
 *   - neighbours are all periodic images with 0 < |r_ij| < r_c (strict);
 *   - W_i^{ab} = sum_j r_ij^a (dU_j/dr_ji)^b (Eq. 6), J^a = sum_b W^{ab} v^b;
 *   - parameter vector z = [w1 (n_neu x N_des, row-major), b1, w2, b2], with the
 *     descriptor order q_0..q_{nR} then q_{nl} with n outer, l inner.
 * Units: eV, Angstrom, amu, fs.
 *
 * Parity-pinned by the CPU test suite (closed forms, finite differences,
 * invariances, brute force).  The SNES rank utilities follow the standard NES
 * rank shaping because the paper defers their values to its reference; they
 * are pinned by their defining properties (sum zero, monotone, the two-member
 * closed form), not by a printed table.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "nep_oracle.h"

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Sizes: Eq. 16 (N_des) and Eq. 26 (N_par).                                 */
/* ------------------------------------------------------------------------ */
int orc_n_des(const orc_hyper* h)
{
    return (h->n_max_R + 1) + (h->n_max_A + 1) * h->l_max;
}

int orc_n_par(const orc_hyper* h)
{
    return (orc_n_des(h) + 2) * h->n_neu + 1;
}

/* index of q_{nl} inside the descriptor vector (n outer, l inner) */
static int idx_nl(const orc_hyper* h, int n, int l)
{
    return (h->n_max_R + 1) + n * h->l_max + (l - 1);
}

/* ------------------------------------------------------------------------ */
/* Chebyshev polynomials of the first and second kind, App. A (Eqs. A1-A3). */
/* T[0..n], U[0..n].                                                         */
/* ------------------------------------------------------------------------ */
void orc_chebyshev(double x, int n, double* T, double* U)
{
    T[0] = 1.0;
    U[0] = 1.0;
    if (n >= 1) {
        T[1] = x;
        U[1] = 2.0 * x;
    }
    for (int k = 2; k <= n; ++k) {
        T[k] = 2.0 * x * T[k - 1] - T[k - 2];
        U[k] = 2.0 * x * U[k - 1] - U[k - 2];
    }
}

/* Cosine cutoff, Eq. 15; zero beyond r_c.  Returns f_c, writes df_c/dr. */
double orc_cutoff(double r, double rc, double* dfc)
{
    if (r > rc) {
        if (dfc) *dfc = 0.0;
        return 0.0;
    }
    if (dfc) *dfc = -0.5 * (ORC_PI / rc) * sin(ORC_PI * r / rc);
    return 0.5 * (1.0 + cos(ORC_PI * r / rc));
}

/*
 * Radial functions g_n(r), n = 0..nmax, Eq. 14, with x = 2(r/r_c - 1)^2 - 1,
 * and their derivatives dg_n/dr using dT_n/dx = n U_{n-1}(x) (Eq. A2).
 */
void orc_radial(double r, double rc, int nmax, double* g, double* dg)
{
    double T[64], U[64];
    double dfc;
    double fc = orc_cutoff(r, rc, &dfc);
    double t = r / rc - 1.0;
    double x = 2.0 * t * t - 1.0;
    double dxdr = 4.0 * t / rc;
    orc_chebyshev(x, nmax, T, U);
    for (int n = 0; n <= nmax; ++n) {
        double dTdx = (n == 0) ? 0.0 : n * U[n - 1];
        g[n] = 0.5 * (T[n] + 1.0) * fc;
        if (dg) dg[n] = 0.5 * dTdx * dxdr * fc + 0.5 * (T[n] + 1.0) * dfc;
    }
}

/*
 * Legendre polynomial P_l(t) by Bonnet's recurrence
 * (k+1) P_{k+1} = (2k+1) t P_k - k P_{k-1}, with its derivative from
 * P'_{k+1} = P'_{k-1} + (2k+1) P_k.
 */
double orc_legendre(int l, double t, double* dP)
{
    double p0 = 1.0, p1 = t;    /* P_{k-1}, P_k  */
    double d0 = 0.0, d1 = 1.0;  /* P'_{k-1}, P'_k */
    if (l == 0) {
        if (dP) *dP = 0.0;
        return 1.0;
    }
    for (int k = 1; k < l; ++k) {
        double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
        double d2 = d0 + (2.0 * k + 1.0) * p1;
        p0 = p1;
        p1 = p2;
        d0 = d1;
        d1 = d2;
    }
    if (dP) *dP = d1;
    return p1;
}

/* ------------------------------------------------------------------------ */
/* Periodic geometry.  box = 3 rows (lattice vectors a, b, c).              */
/* ------------------------------------------------------------------------ */
typedef struct {
    double H[9];     /* rows a, b, c */
    double Hinv[9];  /* inverse: s = r Hinv */
    double d[3];     /* spacing of lattice planes normal to each direction */
} geom;

static int geom_setup(const double* box, geom* G)
{
    const double* a = box;
    const double* b = box + 3;
    const double* c = box + 6;
    double bc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
    double ca[3] = {c[1] * a[2] - c[2] * a[1], c[2] * a[0] - c[0] * a[2], c[0] * a[1] - c[1] * a[0]};
    double ab[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    double vol = a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2];
    if (!(fabs(vol) > 1e-12)) return ORC_ERR_BOX;
    memcpy(G->H, box, 9 * sizeof(double));
    /* H^{-1} columns are the reciprocal vectors bc/vol, ca/vol, ab/vol */
    for (int r = 0; r < 3; ++r) {
        G->Hinv[r * 3 + 0] = bc[r] / vol;
        G->Hinv[r * 3 + 1] = ca[r] / vol;
        G->Hinv[r * 3 + 2] = ab[r] / vol;
    }
    G->d[0] = fabs(vol) / sqrt(bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
    G->d[1] = fabs(vol) / sqrt(ca[0] * ca[0] + ca[1] * ca[1] + ca[2] * ca[2]);
    G->d[2] = fabs(vol) / sqrt(ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2]);
    return ORC_OK;
}

/* fractional coordinates s = r H^{-1}, wrapped into [0, 1) */
static void to_frac_wrapped(const geom* G, const double* r, double* s)
{
    for (int b = 0; b < 3; ++b) {
        double v = r[0] * G->Hinv[0 * 3 + b] + r[1] * G->Hinv[1 * 3 + b] + r[2] * G->Hinv[2 * 3 + b];
        v -= floor(v);
        if (v >= 1.0) v -= 1.0;
        s[b] = v;
    }
}

/* Cartesian vector of a fractional difference */
static void frac_to_cart(const geom* G, const double* ds, double* r)
{
    for (int b = 0; b < 3; ++b) r[b] = ds[0] * G->H[0 * 3 + b] + ds[1] * G->H[1 * 3 + b] + ds[2] * G->H[2 * 3 + b];
}

/* ------------------------------------------------------------------------ */
/* Neighbour lists (CSR).  A pair (i, j, image) is kept when                 */
/* 0 < |r_j + image - r_i| < rc; j == i is allowed for a non-zero image.     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n;
    int* start; /* n + 1 */
    int* j;     /* pair -> neighbour index */
    double* r;  /* pair -> r_ij (3) */
} nlist;

static void nlist_free(nlist* L)
{
    free(L->start);
    free(L->j);
    free(L->r);
    memset(L, 0, sizeof(*L));
}

/* visit all candidate pairs of atom i; mode 0 counts, mode 1 stores */
static int brute_atom(const geom* G, int n, const double* s, double rc, int i, int mode, int* j_out,
                      double* r_out)
{
    int cnt = 0;
    int N[3];
    for (int a = 0; a < 3; ++a) N[a] = (int)ceil(rc / G->d[a]);
    for (int j = 0; j < n; ++j) {
        for (int na = -N[0]; na <= N[0]; ++na)
            for (int nb = -N[1]; nb <= N[1]; ++nb)
                for (int nc = -N[2]; nc <= N[2]; ++nc) {
                    if (j == i && na == 0 && nb == 0 && nc == 0) continue;
                    double ds[3] = {s[3 * j + 0] - s[3 * i + 0] + na, s[3 * j + 1] - s[3 * i + 1] + nb,
                                    s[3 * j + 2] - s[3 * i + 2] + nc};
                    double r[3];
                    frac_to_cart(G, ds, r);
                    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                    if (r2 < rc * rc) {
                        if (mode) {
                            j_out[cnt] = j;
                            r_out[3 * cnt + 0] = r[0];
                            r_out[3 * cnt + 1] = r[1];
                            r_out[3 * cnt + 2] = r[2];
                        }
                        ++cnt;
                    }
                }
    }
    return cnt;
}

/* cell list over the fractional cube; requires >= 3 cells per direction */
typedef struct {
    int nc[3];
    int* cell_start; /* ncell + 1 */
    int* cell_atoms; /* n, atoms ordered by cell, increasing index inside a cell */
} cells;

static int cell_of(const cells* C, const double* s)
{
    int c[3];
    for (int a = 0; a < 3; ++a) {
        c[a] = (int)(s[a] * C->nc[a]);
        if (c[a] >= C->nc[a]) c[a] = C->nc[a] - 1;
        if (c[a] < 0) c[a] = 0;
    }
    return (c[0] * C->nc[1] + c[1]) * C->nc[2] + c[2];
}

static void cells_build(cells* C, int n, const double* s)
{
    int ncell = C->nc[0] * C->nc[1] * C->nc[2];
    C->cell_start = (int*)calloc((size_t)ncell + 1, sizeof(int));
    C->cell_atoms = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) C->cell_start[cell_of(C, s + 3 * i) + 1]++;
    for (int c = 0; c < ncell; ++c) C->cell_start[c + 1] += C->cell_start[c];
    int* fill = (int*)calloc((size_t)ncell, sizeof(int));
    for (int i = 0; i < n; ++i) {
        int c = cell_of(C, s + 3 * i);
        C->cell_atoms[C->cell_start[c] + fill[c]++] = i;
    }
    free(fill);
}

static int cell_atom(const geom* G, const cells* C, const double* s, double rc, int i, int mode, int* j_out,
                     double* r_out)
{
    int cnt = 0;
    int ci[3];
    for (int a = 0; a < 3; ++a) {
        ci[a] = (int)(s[3 * i + a] * C->nc[a]);
        if (ci[a] >= C->nc[a]) ci[a] = C->nc[a] - 1;
    }
    for (int da = -1; da <= 1; ++da)
        for (int db = -1; db <= 1; ++db)
            for (int dc = -1; dc <= 1; ++dc) {
                int cc[3] = {ci[0] + da, ci[1] + db, ci[2] + dc};
                double img[3];
                for (int a = 0; a < 3; ++a) {
                    img[a] = 0.0;
                    if (cc[a] < 0) {
                        cc[a] += C->nc[a];
                        img[a] = -1.0;
                    } else if (cc[a] >= C->nc[a]) {
                        cc[a] -= C->nc[a];
                        img[a] = 1.0;
                    }
                }
                int c = (cc[0] * C->nc[1] + cc[1]) * C->nc[2] + cc[2];
                for (int t = C->cell_start[c]; t < C->cell_start[c + 1]; ++t) {
                    int j = C->cell_atoms[t];
                    if (j == i && img[0] == 0.0 && img[1] == 0.0 && img[2] == 0.0) continue;
                    double ds[3] = {s[3 * j + 0] - s[3 * i + 0] + img[0], s[3 * j + 1] - s[3 * i + 1] + img[1],
                                    s[3 * j + 2] - s[3 * i + 2] + img[2]};
                    double r[3];
                    frac_to_cart(G, ds, r);
                    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                    if (r2 < rc * rc) {
                        if (mode) {
                            j_out[cnt] = j;
                            r_out[3 * cnt + 0] = r[0];
                            r_out[3 * cnt + 1] = r[1];
                            r_out[3 * cnt + 2] = r[2];
                        }
                        ++cnt;
                    }
                }
            }
    return cnt;
}

/* method: 0 = brute force, 1 = cell list (falls back to brute force when a
 * direction holds fewer than 3 cells), 2 = automatic (cell list) */
static int nlist_build(int n, const double* box, const double* pos, double rc, int method, nlist* L)
{
    geom G;
    int rcode = geom_setup(box, &G);
    if (rcode) return rcode;
    memset(L, 0, sizeof(*L));
    L->n = n;
    double* s = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) to_frac_wrapped(&G, pos + 3 * i, s + 3 * i);

    cells C;
    memset(&C, 0, sizeof(C));
    int use_cells = (method != 0);
    for (int a = 0; a < 3; ++a) {
        C.nc[a] = (int)floor(G.d[a] / rc);
        if (C.nc[a] < 3) use_cells = 0;
    }
    if (use_cells) cells_build(&C, n, s);

    L->start = (int*)calloc((size_t)n + 1, sizeof(int));
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i)
        L->start[i + 1] = use_cells ? cell_atom(&G, &C, s, rc, i, 0, NULL, NULL) : brute_atom(&G, n, s, rc, i, 0, NULL, NULL);
    for (int i = 0; i < n; ++i) L->start[i + 1] += L->start[i];
    size_t np = (size_t)L->start[n];
    L->j = (int*)malloc(sizeof(int) * (np > 0 ? np : 1));
    L->r = (double*)malloc(sizeof(double) * 3 * (np > 0 ? np : 1));
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        int o = L->start[i];
        if (use_cells)
            cell_atom(&G, &C, s, rc, i, 1, L->j + o, L->r + 3 * (size_t)o);
        else
            brute_atom(&G, n, s, rc, i, 1, L->j + o, L->r + 3 * (size_t)o);
    }
    if (use_cells) {
        free(C.cell_start);
        free(C.cell_atoms);
    }
    free(s);
    return ORC_OK;
}

int orc_neighbors(int n, const double* box, const double* pos, double rc, int method, int cap, int* count,
                  int* nbr_j, double* nbr_r)
{
    nlist L;
    int rcode = nlist_build(n, box, pos, rc, method, &L);
    if (rcode) return rcode;
    int over = 0;
    for (int i = 0; i < n; ++i) {
        int m = L.start[i + 1] - L.start[i];
        count[i] = m;
        if (m > cap) {
            over = 1;
            m = cap;
        }
        for (int t = 0; t < m; ++t) {
            nbr_j[(size_t)i * cap + t] = L.j[L.start[i] + t];
            for (int a = 0; a < 3; ++a) nbr_r[((size_t)i * cap + t) * 3 + a] = L.r[3 * (size_t)(L.start[i] + t) + a];
        }
    }
    nlist_free(&L);
    return over ? ORC_ERR_CAPACITY : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Per-atom environment quantities.                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int m;
    const double* r;  /* m x 3, r_ij */
    double* rn;       /* m, |r_ij| */
    double* gR;       /* m x (nR+1) */
    double* dgR;
    double* gA;       /* m x (nA+1) */
    double* dgA;
} env;

/*
 * Multicomponent weighting (Sec. II.A, "Multicomponent systems"): the cutoff
 * function of pair (i, j) becomes f_c(r_ij) sqrt(Z_i Z_j); since g_n and g_n'
 * are linear in f_c, both are multiplied by w_ij = sqrt(Z_i Z_j).  Zat holds
 * the Z of every atom of the call (NULL: one species, w = 1); jlist the
 * neighbours of atom i.
 */
static void env_fill(const orc_hyper* h, env* E, const double* Zat, int i, const int* jlist)
{
    int nR = h->n_max_R + 1, nA = h->n_max_A + 1;
    for (int a = 0; a < E->m; ++a) {
        const double* v = E->r + 3 * a;
        double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        E->rn[a] = r;
        const double w = Zat ? sqrt(Zat[i] * Zat[jlist[a]]) : 1.0;
        if (r < h->rc_R)
            orc_radial(r, h->rc_R, h->n_max_R, E->gR + a * nR, E->dgR + a * nR);
        else
            for (int n = 0; n < nR; ++n) E->gR[a * nR + n] = E->dgR[a * nR + n] = 0.0;
        if (r < h->rc_A)
            orc_radial(r, h->rc_A, h->n_max_A, E->gA + a * nA, E->dgA + a * nA);
        else
            for (int n = 0; n < nA; ++n) E->gA[a * nA + n] = E->dgA[a * nA + n] = 0.0;
        for (int n = 0; n < nR; ++n) {
            E->gR[a * nR + n] *= w;
            E->dgR[a * nR + n] *= w;
        }
        for (int n = 0; n < nA; ++n) {
            E->gA[a * nA + n] *= w;
            E->dgA[a * nA + n] *= w;
        }
    }
}

static void env_alloc(const orc_hyper* h, env* E, int m, const double* r, const double* Zat, int i,
                      const int* jlist)
{
    int nR = h->n_max_R + 1, nA = h->n_max_A + 1;
    int mm = m > 0 ? m : 1;
    E->m = m;
    E->r = r;
    E->rn = (double*)malloc(sizeof(double) * mm);
    E->gR = (double*)malloc(sizeof(double) * mm * nR);
    E->dgR = (double*)malloc(sizeof(double) * mm * nR);
    E->gA = (double*)malloc(sizeof(double) * mm * nA);
    E->dgA = (double*)malloc(sizeof(double) * mm * nA);
    env_fill(h, E, Zat, i, jlist);
}

static void env_free(env* E)
{
    free(E->rn);
    free(E->gR);
    free(E->dgR);
    free(E->gA);
    free(E->dgA);
}

static double cos_angle(const env* E, int a, int b)
{
    const double* u = E->r + 3 * a;
    const double* v = E->r + 3 * b;
    return (u[0] * v[0] + u[1] * v[1] + u[2] * v[2]) / (E->rn[a] * E->rn[b]);
}

/* Descriptor of one atom: radial part Eq. 12, angular part Eq. 13 as the
 * literal double sum over neighbour pairs (j, k), k = j included. */
static void descriptor(const orc_hyper* h, const env* E, double* q)
{
    int nR = h->n_max_R + 1, nA = h->n_max_A + 1;
    int nd = orc_n_des(h);
    for (int v = 0; v < nd; ++v) q[v] = 0.0;
    for (int a = 0; a < E->m; ++a)
        if (E->rn[a] < h->rc_R)
            for (int n = 0; n < nR; ++n) q[n] += E->gR[a * nR + n];
    for (int a = 0; a < E->m; ++a) {
        if (!(E->rn[a] < h->rc_A)) continue;
        for (int b = 0; b < E->m; ++b) {
            if (!(E->rn[b] < h->rc_A)) continue;
            double c = cos_angle(E, a, b);
            for (int l = 1; l <= h->l_max; ++l) {
                double P = orc_legendre(l, c, NULL);
                for (int n = 0; n < nA; ++n) q[idx_nl(h, n, l)] += E->gA[a * nA + n] * E->gA[b * nA + n] * P;
            }
        }
    }
}

/* Network of Eqs. 21-22: site energy U, hidden state x, and G = dU/dq. */
static double network(const orc_hyper* h, const double* z, const double* q, double* x, double* G)
{
    int nd = orc_n_des(h), nh = h->n_neu;
    const double* w1 = z;
    const double* b1 = z + nh * nd;
    const double* w2 = b1 + nh;
    double b2 = w2[nh];
    double U = 0.0;
    for (int mu = 0; mu < nh; ++mu) {
        double a = 0.0;
        for (int v = 0; v < nd; ++v) a += w1[mu * nd + v] * q[v];
        x[mu] = tanh(a - b1[mu]);
        U += w2[mu] * x[mu];
    }
    U -= b2;
    if (G) {
        for (int v = 0; v < nd; ++v) G[v] = 0.0;
        for (int mu = 0; mu < nh; ++mu) {
            double c = w2[mu] * (1.0 - x[mu] * x[mu]);
            for (int v = 0; v < nd; ++v) G[v] += c * w1[mu * nd + v];
        }
    }
    return U;
}

/*
 * Derivatives of every descriptor component of atom i with respect to r_ij
 * for neighbour a (= j): Eq. 24 (radial) and Eq. 25 (angular).
 * J is N_des x 3.
 */
static void descriptor_jacobian(const orc_hyper* h, const env* E, int a, double* J)
{
    int nR = h->n_max_R + 1, nA = h->n_max_A + 1;
    int nd = orc_n_des(h);
    for (int v = 0; v < 3 * nd; ++v) J[v] = 0.0;
    double ra = E->rn[a];
    double ua[3] = {E->r[3 * a] / ra, E->r[3 * a + 1] / ra, E->r[3 * a + 2] / ra};
    if (ra < h->rc_R)
        for (int n = 0; n < nR; ++n)
            for (int c = 0; c < 3; ++c) J[n * 3 + c] = E->dgR[a * nR + n] * ua[c];
    if (!(ra < h->rc_A)) return;
    for (int b = 0; b < E->m; ++b) {
        if (!(E->rn[b] < h->rc_A)) continue;
        double rb = E->rn[b];
        double ub[3] = {E->r[3 * b] / rb, E->r[3 * b + 1] / rb, E->r[3 * b + 2] / rb};
        double cth = cos_angle(E, a, b);
        for (int l = 1; l <= h->l_max; ++l) {
            double dP;
            double P = orc_legendre(l, cth, &dP);
            for (int n = 0; n < nA; ++n) {
                double t1 = 2.0 * E->dgA[a * nA + n] * E->gA[b * nA + n] * P;
                double t2 = 2.0 * E->gA[a * nA + n] * E->gA[b * nA + n] * dP / ra;
                int v = idx_nl(h, n, l);
                for (int c = 0; c < 3; ++c) J[v * 3 + c] += t1 * ua[c] + t2 * (ub[c] - ua[c] * cth);
            }
        }
    }
}

/* Partial force dU_i/dr_ij = sum_nu G_nu dq_nu/dr_ij, Eq. 23. */
static void partial_force(const orc_hyper* h, const env* E, int a, const double* G, double* Jbuf, double* p)
{
    int nd = orc_n_des(h);
    descriptor_jacobian(h, E, a, Jbuf);
    p[0] = p[1] = p[2] = 0.0;
    for (int v = 0; v < nd; ++v)
        for (int c = 0; c < 3; ++c) p[c] += G[v] * Jbuf[v * 3 + c];
}

static double max_cutoff(const orc_hyper* h)
{
    return h->rc_R > h->rc_A ? h->rc_R : h->rc_A;
}

static int check_hyper(const orc_hyper* h)
{
    if (h->n_max_R < 0 || h->n_max_R > 60 || h->n_max_A < 0 || h->n_max_A > 60 || h->l_max < 1 || h->l_max > 8 ||
        h->n_neu < 1 || !(h->rc_R > 0) || !(h->rc_A > 0))
        return ORC_ERR_ARG;
    return ORC_OK;
}

int orc_descriptors(const orc_hyper* h, int n, const double* box, const double* pos, double* q)
{
    return orc_descriptors_z(h, n, box, pos, NULL, q);
}

/* orc_descriptors with per-atom atomic numbers Zat (n), the multicomponent weighting */
int orc_descriptors_z(const orc_hyper* h, int n, const double* box, const double* pos, const double* Zat, double* q)
{
    int rcode = check_hyper(h);
    if (rcode) return rcode;
    nlist L;
    rcode = nlist_build(n, box, pos, max_cutoff(h), 2, &L);
    if (rcode) return rcode;
    int nd = orc_n_des(h);
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        env E;
        env_alloc(h, &E, L.start[i + 1] - L.start[i], L.r + 3 * (size_t)L.start[i], Zat, i, L.j + L.start[i]);
        descriptor(h, &E, q + (size_t)i * nd);
        env_free(&E);
    }
    nlist_free(&L);
    return ORC_OK;
}

/*
 * Energy, forces and per-atom virial.
 *   U[i]      site energy (Eq. 22)
 *   F[3i+a]   F_i = sum_j (dU_i/dr_ij - dU_j/dr_ji)        (Eqs. 4-5)
 *   W[9i+3a+b] = sum_j r_ij^a (dU_j/dr_ji)^b              (Eq. 6)
 * Any output pointer may be NULL.  q (n x N_des), G (n x N_des) and
 * x (n x n_neu) are optional intermediate outputs.
 */
static int efv_impl(const orc_hyper* h, const double* z, int n, const double* box, const double* pos,
                    int nlist_method, const double* Zat, double* U, double* F, double* W, double* q_out,
                    double* G_out, double* x_out)
{
    int rcode = check_hyper(h);
    if (rcode) return rcode;
    nlist L;
    rcode = nlist_build(n, box, pos, max_cutoff(h), nlist_method, &L);
    if (rcode) return rcode;
    int nd = orc_n_des(h), nh = h->n_neu;
    size_t np = (size_t)L.start[n];
    double* p = (double*)malloc(sizeof(double) * 3 * (np > 0 ? np : 1));

#pragma omp parallel
    {
        double* q = (double*)malloc(sizeof(double) * nd);
        double* G = (double*)malloc(sizeof(double) * nd);
        double* x = (double*)malloc(sizeof(double) * nh);
        double* Jb = (double*)malloc(sizeof(double) * 3 * nd);
#pragma omp for schedule(dynamic, 16)
        for (int i = 0; i < n; ++i) {
            env E;
            env_alloc(h, &E, L.start[i + 1] - L.start[i], L.r + 3 * (size_t)L.start[i], Zat, i, L.j + L.start[i]);
            descriptor(h, &E, q);
            double Ui = network(h, z, q, x, G);
            if (U) U[i] = Ui;
            if (q_out) memcpy(q_out + (size_t)i * nd, q, sizeof(double) * nd);
            if (G_out) memcpy(G_out + (size_t)i * nd, G, sizeof(double) * nd);
            if (x_out) memcpy(x_out + (size_t)i * nh, x, sizeof(double) * nh);
            for (int a = 0; a < E.m; ++a) partial_force(h, &E, a, G, Jb, p + 3 * ((size_t)L.start[i] + a));
            env_free(&E);
        }
        free(q);
        free(G);
        free(x);
        free(Jb);
    }

    /* assemble in a fixed serial order: every stored pair (i -> j) adds its
     * partial force to F_i, subtracts it from F_j, and adds r_ji (x) p_ij to W_j */
    if (F) memset(F, 0, sizeof(double) * 3 * (size_t)n);
    if (W) memset(W, 0, sizeof(double) * 9 * (size_t)n);
    for (int i = 0; i < n; ++i)
        for (int t = L.start[i]; t < L.start[i + 1]; ++t) {
            int j = L.j[t];
            const double* pij = p + 3 * (size_t)t;
            const double* rij = L.r + 3 * (size_t)t;
            if (F)
                for (int c = 0; c < 3; ++c) {
                    F[3 * (size_t)i + c] += pij[c];
                    F[3 * (size_t)j + c] -= pij[c];
                }
            if (W)
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) W[9 * (size_t)j + 3 * a + b] += -rij[a] * pij[b];
        }
    free(p);
    nlist_free(&L);
    return ORC_OK;
}

int orc_efv(const orc_hyper* h, const double* z, int n, const double* box, const double* pos, double* U, double* F,
            double* W)
{
    return efv_impl(h, z, n, box, pos, 2, NULL, U, F, W, NULL, NULL, NULL);
}

/* orc_efv with per-atom atomic numbers Zat (n), the multicomponent weighting */
int orc_efv_z(const orc_hyper* h, const double* z, int n, const double* box, const double* pos, const double* Zat,
              double* U, double* F, double* W)
{
    return efv_impl(h, z, n, box, pos, 2, Zat, U, F, W, NULL, NULL, NULL);
}

int orc_efv_brute(const orc_hyper* h, const double* z, int n, const double* box, const double* pos, double* U,
                  double* F, double* W)
{
    return efv_impl(h, z, n, box, pos, 0, NULL, U, F, W, NULL, NULL, NULL);
}

int orc_site(const orc_hyper* h, const double* z, int n, const double* box, const double* pos, double* q,
             double* G, double* x)
{
    return efv_impl(h, z, n, box, pos, 2, NULL, NULL, NULL, NULL, q, G, x);
}

/*
 * Energy, force and per-atom virial of selected atoms only (same definitions
 * as orc_efv).  Site quantities are evaluated for the selected atoms and their
 * neighbours; F_i and W_i need the neighbours' partial forces towards i,
 * found as the neighbour's pair with the opposite vector.
 */
int orc_efv_sample(const orc_hyper* h, const double* z, int n, const double* box, const double* pos, int n_sample,
                   const int* idx, double* U, double* F, double* W)
{
    const double* Zat = NULL; /* one species */
    int rcode = check_hyper(h);
    if (rcode) return rcode;
    nlist L;
    rcode = nlist_build(n, box, pos, max_cutoff(h), 2, &L);
    if (rcode) return rcode;
    int nd = orc_n_des(h), nh = h->n_neu;
    char* need = (char*)calloc((size_t)n, 1);
    for (int s = 0; s < n_sample; ++s) {
        int i = idx[s];
        if (i < 0 || i >= n) {
            free(need);
            nlist_free(&L);
            return ORC_ERR_ARG;
        }
        need[i] = 1;
        for (int t = L.start[i]; t < L.start[i + 1]; ++t) need[L.j[t]] = 1;
    }
    size_t np = (size_t)L.start[n];
    double* p = (double*)calloc(3 * (np > 0 ? np : 1), sizeof(double));
    double* Ua = (double*)calloc((size_t)n, sizeof(double));
#pragma omp parallel
    {
        double* q = (double*)malloc(sizeof(double) * nd);
        double* G = (double*)malloc(sizeof(double) * nd);
        double* x = (double*)malloc(sizeof(double) * nh);
        double* Jb = (double*)malloc(sizeof(double) * 3 * nd);
#pragma omp for schedule(dynamic, 16)
        for (int i = 0; i < n; ++i) {
            if (!need[i]) continue;
            env E;
            env_alloc(h, &E, L.start[i + 1] - L.start[i], L.r + 3 * (size_t)L.start[i], Zat, i, L.j + L.start[i]);
            descriptor(h, &E, q);
            Ua[i] = network(h, z, q, x, G);
            for (int a = 0; a < E.m; ++a) partial_force(h, &E, a, G, Jb, p + 3 * ((size_t)L.start[i] + a));
            env_free(&E);
        }
        free(q);
        free(G);
        free(x);
        free(Jb);
    }
    for (int s = 0; s < n_sample; ++s) {
        int i = idx[s];
        if (U) U[s] = Ua[i];
        double f[3] = {0, 0, 0}, w[9] = {0};
        for (int t = L.start[i]; t < L.start[i + 1]; ++t) {
            int j = L.j[t];
            const double* rij = L.r + 3 * (size_t)t;
            /* the pair of j pointing back to i through the opposite image */
            int back = -1;
            for (int u = L.start[j]; u < L.start[j + 1]; ++u) {
                const double* rji = L.r + 3 * (size_t)u;
                if (L.j[u] == i && fabs(rji[0] + rij[0]) < 1e-9 && fabs(rji[1] + rij[1]) < 1e-9 &&
                    fabs(rji[2] + rij[2]) < 1e-9) {
                    back = u;
                    break;
                }
            }
            const double* pij = p + 3 * (size_t)t;
            for (int c = 0; c < 3; ++c) f[c] += pij[c];
            if (back >= 0) {
                const double* pji = p + 3 * (size_t)back;
                for (int c = 0; c < 3; ++c) f[c] -= pji[c];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) w[3 * a + b] += rij[a] * pji[b];
            }
        }
        if (F) memcpy(F + 3 * (size_t)s, f, sizeof(f));
        if (W) memcpy(W + 9 * (size_t)s, w, sizeof(w));
    }
    free(p);
    free(Ua);
    free(need);
    nlist_free(&L);
    return ORC_OK;
}

/* Heat current J = sum_i W_i . v_i (Eq. 7), J^a = sum_b W_i^{ab} v_i^b. */
void orc_heat_current(int n, const double* W, const double* v, double* J)
{
    J[0] = J[1] = J[2] = 0.0;
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) J[a] += W[9 * (size_t)i + 3 * a + b] * v[3 * (size_t)i + b];
}

/* ------------------------------------------------------------------------ */
/* NVE velocity-Verlet molecular dynamics.                                   */
/* ------------------------------------------------------------------------ */
/* 1 amu * A^2 / fs^2 expressed in eV (CODATA 2018 amu and elementary charge) */
static double amu_a2_fs2_in_ev(void)
{
    return 1.66053906660e-27 * 1.0e-20 / 1.0e-30 / 1.602176634e-19;
}

/*
 * n_steps of velocity Verlet with time step dt (fs) and one mass (amu).
 * Per step: v += dt/2 F/m; x += dt v; F = F(x); v += dt/2 F/m; then the heat
 * current J = sum_i W_i v_i is taken with the new W and v.
 * thermo (n_steps x 2): potential energy, kinetic energy (eV).  J (n_steps x 3).
 * Positions are not wrapped.
 */
int orc_md(const orc_hyper* h, const double* z, int n, const double* box, double* pos, double* vel, double mass,
           double dt, int n_steps, double* thermo, double* J)
{
    double conv = amu_a2_fs2_in_ev();
    double* U = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* F = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double* W = (double*)malloc(sizeof(double) * 9 * (size_t)(n > 0 ? n : 1));
    int rcode = orc_efv(h, z, n, box, pos, U, F, W);
    double acc = dt * 0.5 / (mass * conv);
    for (int s = 0; s < n_steps && !rcode; ++s) {
        for (int k = 0; k < 3 * n; ++k) {
            vel[k] += acc * F[k];
            pos[k] += dt * vel[k];
        }
        rcode = orc_efv(h, z, n, box, pos, U, F, W);
        if (rcode) break;
        for (int k = 0; k < 3 * n; ++k) vel[k] += acc * F[k];
        double ep = 0.0, ek = 0.0;
        for (int i = 0; i < n; ++i) ep += U[i];
        for (int k = 0; k < 3 * n; ++k) ek += 0.5 * mass * conv * vel[k] * vel[k];
        if (thermo) {
            thermo[2 * s + 0] = ep;
            thermo[2 * s + 1] = ek;
        }
        if (J) orc_heat_current(n, W, vel, J + 3 * s);
    }
    free(U);
    free(F);
    free(W);
    return rcode;
}

/*
 * The same integrator with two optional extensions for heat transport:
 *   HNEMD driving (Sec. II.B): every atom feels F_i^ext = F_e . W_i, i.e.
 *     (F_i^ext)^b = sum_a F_e^a W_i^{ab}, minus the mean over all atoms so that
 *     the total momentum is kept (fe = NULL or zero: off);
 *   Berendsen thermostat: after the second half kick and the heat current,
 *     v *= lambda with lambda^2 = 1 + (dt/tau)(T0/T - 1), T = 2 E_kin /
 *     ((3N - 3) k_B) (tau <= 0: off).
 * Per step: v += dt/2 F/m; x += dt v; F = F_NEP(x) + F_ext; v += dt/2 F/m;
 * J = sum_i W_i v_i; thermostat.  thermo (n_steps x 2): potential energy and
 * kinetic energy after the thermostat.  J (n_steps x 3): before it.
 * With fe = NULL and tau <= 0 this is orc_md step for step.
 */
int orc_md_ext(const orc_hyper* h, const double* z, int n, const double* box, double* pos, double* vel,
               double mass, double dt, int n_steps, double t0, double tau, const double* fe, double* thermo,
               double* J)
{
    return orc_md_record(h, z, n, box, pos, vel, mass, dt, n_steps, t0, tau, fe, NULL, thermo, J, NULL, NULL);
}

/*
 * orc_md_ext that also records, for every step s, the per-atom virials W_i
 * (n x 9) and velocities v_i (n x 3) from which J(s) is taken (after the
 * second half kick, before the thermostat): W_hist[s], v_hist[s].  Zat: the
 * atomic number of every atom (multicomponent weighting), or NULL.
 */
int orc_md_record(const orc_hyper* h, const double* z, int n, const double* box, double* pos, double* vel,
                  double mass, double dt, int n_steps, double t0, double tau, const double* fe, const double* Zat,
                  double* thermo, double* J, double* W_hist, double* v_hist)
{
    const double conv = amu_a2_fs2_in_ev();
    const double kb = 8.617333262e-5; /* eV/K, CODATA 2018 */
    double* U = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* F = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double* W = (double*)malloc(sizeof(double) * 9 * (size_t)(n > 0 ? n : 1));
    const int drive = fe && (fe[0] != 0.0 || fe[1] != 0.0 || fe[2] != 0.0);
    int rcode = orc_efv_z(h, z, n, box, pos, Zat, U, F, W);
    const double acc = dt * 0.5 / (mass * conv);
    for (int s = -1; s < n_steps && !rcode; ++s) {
        if (s >= 0) {
            for (int k = 0; k < 3 * n; ++k) {
                vel[k] += acc * F[k];
                pos[k] += dt * vel[k];
            }
            rcode = orc_efv_z(h, z, n, box, pos, Zat, U, F, W);
            if (rcode) break;
        }
        if (drive) {
            double mean[3] = {0.0, 0.0, 0.0};
            double* fx = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
            for (int i = 0; i < n; ++i)
                for (int b = 0; b < 3; ++b) {
                    double f = 0.0;
                    for (int a = 0; a < 3; ++a) f += fe[a] * W[9 * (size_t)i + 3 * a + b];
                    fx[3 * (size_t)i + b] = f;
                    mean[b] += f;
                }
            for (int b = 0; b < 3; ++b) mean[b] /= (double)n;
            for (int i = 0; i < n; ++i)
                for (int b = 0; b < 3; ++b) F[3 * (size_t)i + b] += fx[3 * (size_t)i + b] - mean[b];
            free(fx);
        }
        if (s < 0) continue; /* forces of the starting configuration */
        for (int k = 0; k < 3 * n; ++k) vel[k] += acc * F[k];
        if (J) orc_heat_current(n, W, vel, J + 3 * s);
        if (W_hist) memcpy(W_hist + (size_t)s * 9 * n, W, sizeof(double) * 9 * (size_t)n);
        if (v_hist) memcpy(v_hist + (size_t)s * 3 * n, vel, sizeof(double) * 3 * (size_t)n);
        double ep = 0.0, ek = 0.0;
        for (int i = 0; i < n; ++i) ep += U[i];
        for (int k = 0; k < 3 * n; ++k) ek += 0.5 * mass * conv * vel[k] * vel[k];
        if (tau > 0.0 && n > 1 && ek > 0.0) {
            const double T = 2.0 * ek / ((3.0 * n - 3.0) * kb);
            const double lam = sqrt(1.0 + dt / tau * (t0 / T - 1.0));
            for (int k = 0; k < 3 * n; ++k) vel[k] *= lam;
            ek *= lam * lam;
        }
        if (thermo) {
            thermo[2 * s + 0] = ep;
            thermo[2 * s + 1] = ek;
        }
    }
    free(U);
    free(F);
    free(W);
    return rcode;
}

/* ------------------------------------------------------------------------ */
/* Spectral heat current (Sec. II.B).                                        */
/* ------------------------------------------------------------------------ */
/*
 * Virial-velocity correlation K(t) = sum_i < W_i(0) . v_i(t) >, with
 * (W . v)^a = sum_b W^{ab} v^b (the contraction of the heat current, Eq. 7).
 * Given the per-atom virials and velocities of n_samples samples taken dt_s
 * apart (W_hist[s] n x 9, v_hist[s] n x 3), K_sum[tau][a] is the sum over all
 * time origins s0 with s0 + tau < n_samples of sum_i (W_i(s0) . v_i(s0 + tau))^a,
 * for 0 <= tau < n_lags; the average is K_sum[tau] / (n_samples - tau).
 */
void orc_shc(int n, int n_samples, int n_lags, const double* W_hist, const double* v_hist, double* K_sum)
{
    for (int t = 0; t < n_lags; ++t)
        for (int a = 0; a < 3; ++a) K_sum[3 * t + a] = 0.0;
    for (int s = 0; s < n_samples; ++s) {          /* the later time s0 + tau */
        const double* v = v_hist + (size_t)s * 3 * n;
        for (int t = 0; t < n_lags && t <= s; ++t) {  /* lag tau: origin s - tau */
            const double* W = W_hist + (size_t)(s - t) * 9 * n;
            for (int i = 0; i < n; ++i)
                for (int a = 0; a < 3; ++a) {
                    double k = 0.0;
                    for (int b = 0; b < 3; ++b) k += W[9 * (size_t)i + 3 * a + b] * v[3 * (size_t)i + b];
                    K_sum[3 * t + a] += k;
                }
        }
    }
}

/*
 * The transform of Sec. II.B: (2 / (T V)) int K(t) e^{i w t} dt =
 * sum_nu kappa_{mu nu}(w) F_e^nu.  K is known at t = tau dt_s for
 * 0 <= tau < n_lags and taken as even in t (steady state), so the integral is
 * 2 int_0^T K(t) cos(w t) dt with T = (n_lags - 1) dt_s, evaluated by the
 * trapezoid rule; window = 1 multiplies K by the Hann window
 * (1 + cos(pi tau / (n_lags - 1))) / 2 first.  out[k][a] = scale * integral
 * for omega[k] (rad per unit of dt_s); scale = 2 / (T V F_e) gives kappa(w).
 */
void orc_shc_spectrum(int n_lags, const double* K, double dt_s, int n_omega, const double* omega, double scale,
                      int window, double* out)
{
    for (int k = 0; k < n_omega; ++k)
        for (int a = 0; a < 3; ++a) {
            double sum = 0.0;
            for (int t = 0; t < n_lags; ++t) {
                double w = (t == 0 || t == n_lags - 1) ? 0.5 : 1.0; /* trapezoid weights */
                if (window && n_lags > 1) w *= 0.5 * (1.0 + cos(ORC_PI * t / (n_lags - 1)));
                sum += w * K[3 * t + a] * cos(omega[k] * t * dt_s);
            }
            out[3 * k + a] = scale * 2.0 * dt_s * sum;
        }
}

/*
 * Quantum correction of a classical spectral conductivity (Sec. IV.C):
 * kappa_q(w) = kappa(w) x^2 e^x / (e^x - 1)^2 with x = hbar w / (k_B T),
 * here x = x_per_omega * omega[k].  The factor is the paper's with numerator
 * and denominator multiplied by e^{-2x}, x^2 e^{-x} / (1 - e^{-x})^2, so that
 * e^x cannot overflow, and expm1 for the denominator; its limit 1 at x = 0.
 * spec [n_omega][3] is scaled in place.
 */
void orc_shc_quantum(int n_omega, const double* omega, double x_per_omega, double* spec)
{
    for (int k = 0; k < n_omega; ++k) {
        const double x = fabs(x_per_omega * omega[k]);
        double f = 1.0;
        if (x > 0.0) {
            const double em = -expm1(-x); /* 1 - e^{-x} */
            f = x * x * exp(-x) / (em * em);
        }
        for (int a = 0; a < 3; ++a) spec[3 * k + a] *= f;
    }
}

/*
 * Running HNEMD conductivity estimate (Sec. II.B): <J>/(T V) = kappa F_e, so
 * with scale = 1 / (T V F_e) the estimate after step t is scale times the
 * mean of J over steps 0..t.  J [n][3]; out [n][3]; the sums run in step
 * order.
 */
void orc_hnemd_kappa(int n, const double* J, double scale, double* out)
{
    double sum[3] = {0.0, 0.0, 0.0};
    for (int t = 0; t < n; ++t)
        for (int a = 0; a < 3; ++a) {
            sum[a] += J[3 * t + a];
            out[3 * t + a] = scale * sum[a] / (double)(t + 1);
        }
}

/* ------------------------------------------------------------------------ */
/* Loss function, Eqs. 29-34.                                                */
/* ------------------------------------------------------------------------ */
/*
 * Dataset: n_struct structures; structure s has n_atoms[s] atoms whose
 * positions are the next n_atoms[s] rows of pos (x 3), box boxes[9 s].
 * e_tar: total energy per structure; f_tar: per atom (x 3);
 * w_tar: six virial components per structure in the order xx yy zz xy yz zx,
 * with the virial W = sum_i W_i.
 * Energy and virial enter per atom (divided by the structure's atom count).
 * lambdas = {l_e, l_f, l_v, l_1, l_2}.  out = {L, L_e, L_f, L_v, L_1, L_2}.
 */
static const int VIR6[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {1, 2}, {2, 0}};

int orc_loss(const orc_hyper* h, const double* z, int n_struct, const int* n_atoms, const double* boxes,
             const double* pos, const double* e_tar, const double* f_tar, const double* w_tar,
             const double* lambdas, double* out)
{
    return orc_loss_z(h, z, n_struct, n_atoms, boxes, pos, NULL, e_tar, f_tar, w_tar, lambdas, out);
}

/* orc_loss with the atomic number of every atom of the set (Zat, concatenated like pos) */
int orc_loss_z(const orc_hyper* h, const double* z, int n_struct, const int* n_atoms, const double* boxes,
               const double* pos, const double* Zat, const double* e_tar, const double* f_tar,
               const double* w_tar, const double* lambdas, double* out)
{
    int npar = orc_n_par(h);
    double se = 0.0, sf = 0.0, sv = 0.0;
    long ntot = 0;
    size_t off = 0;
    int rcode = ORC_OK;
    for (int s = 0; s < n_struct && !rcode; ++s) {
        int na = n_atoms[s];
        double* U = (double*)malloc(sizeof(double) * na);
        double* F = (double*)malloc(sizeof(double) * 3 * na);
        double* W = (double*)malloc(sizeof(double) * 9 * na);
        rcode = orc_efv_z(h, z, na, boxes + 9 * s, pos + 3 * off, Zat ? Zat + off : NULL, U, F, W);
        if (!rcode) {
            double E = 0.0, Wt[9] = {0};
            for (int i = 0; i < na; ++i) {
                E += U[i];
                for (int c = 0; c < 9; ++c) Wt[c] += W[9 * i + c];
            }
            double de = (E - e_tar[s]) / na;
            se += de * de;
            for (int k = 0; k < 3 * na; ++k) {
                double d = F[k] - f_tar[3 * off + k];
                sf += d * d;
            }
            for (int c = 0; c < 6; ++c) {
                double d = (Wt[3 * VIR6[c][0] + VIR6[c][1]] - w_tar[6 * s + c]) / na;
                sv += d * d;
            }
        }
        ntot += na;
        off += na;
        free(U);
        free(F);
        free(W);
    }
    if (rcode) return rcode;
    double l1 = 0.0, l2 = 0.0;
    for (int k = 0; k < npar; ++k) {
        l1 += fabs(z[k]);
        l2 += z[k] * z[k];
    }
    out[1] = sqrt(se / n_struct);
    out[2] = sqrt(sf / (3.0 * ntot));
    out[3] = sqrt(sv / (6.0 * n_struct));
    out[4] = l1 / npar;
    out[5] = sqrt(l2 / npar);
    out[0] = lambdas[0] * out[1] + lambdas[1] * out[2] + lambdas[2] * out[3] + lambdas[3] * out[4] +
             lambdas[4] * out[5];
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Gradient of the force loss L_f (Eq. 31) with respect to z, by the chain   */
/* rule through the partial forces (Eqs. 21-25).  Not in the paper (its      */
/* training is gradient-free); written directly from those equations:        */
/*   dL_f/dF_i = (F_i - F_i^tar) / (3 N L_f) =: dF_i                         */
/*   lambda_i,nu = sum_j dq_i,nu/dr_ij . (dF_i - dF_j)                       */
/*   s_mu = sum_nu w1_mu,nu lambda_nu                                        */
/*   dL/dw2_mu = (1 - x_mu^2) s_mu                                           */
/*   dL/db1_mu = 2 w2_mu x_mu (1 - x_mu^2) s_mu                              */
/*   dL/dw1_mu,k = w2_mu (1 - x_mu^2) lambda_k - 2 w2_mu x_mu (1-x_mu^2) s_mu q_k */
/*   dL/db2 = 0,  summed over atoms of all structures.                       */
/* Returns L_f in *lf.                                                       */
/* ------------------------------------------------------------------------ */
int orc_force_loss_grad(const orc_hyper* h, const double* z, int n_struct, const int* n_atoms,
                        const double* boxes, const double* pos, const double* f_tar, double* grad, double* lf)
{
    return orc_force_loss_grad_z(h, z, n_struct, n_atoms, boxes, pos, NULL, f_tar, grad, lf);
}

/* orc_force_loss_grad with the atomic number of every atom (Zat, concatenated like pos) */
int orc_force_loss_grad_z(const orc_hyper* h, const double* z, int n_struct, const int* n_atoms,
                          const double* boxes, const double* pos, const double* Zat, const double* f_tar,
                          double* grad, double* lf)
{
    int rcode = check_hyper(h);
    if (rcode) return rcode;
    int nd = orc_n_des(h), nh = h->n_neu, npar = orc_n_par(h);
    const double* w1 = z;
    const double* w2 = z + nh * nd + nh;
    long ntot = 0;
    for (int s = 0; s < n_struct; ++s) ntot += n_atoms[s];

    /* forward pass: forces of all structures, to get L_f */
    double* Fall = (double*)malloc(sizeof(double) * 3 * (size_t)(ntot > 0 ? ntot : 1));
    size_t off = 0;
    for (int s = 0; s < n_struct; ++s) {
        rcode = orc_efv_z(h, z, n_atoms[s], boxes + 9 * s, pos + 3 * off, Zat ? Zat + off : NULL, NULL,
                          Fall + 3 * off, NULL);
        if (rcode) {
            free(Fall);
            return rcode;
        }
        off += n_atoms[s];
    }
    double sf = 0.0;
    for (long k = 0; k < 3 * ntot; ++k) sf += (Fall[k] - f_tar[k]) * (Fall[k] - f_tar[k]);
    double L = sqrt(sf / (3.0 * ntot));
    if (lf) *lf = L;
    for (int k = 0; k < npar; ++k) grad[k] = 0.0;
    if (!(L > 0.0)) {
        free(Fall);
        return ORC_OK;
    }

    off = 0;
    for (int s = 0; s < n_struct && !rcode; ++s) {
        int na = n_atoms[s];
        nlist Lst;
        rcode = nlist_build(na, boxes + 9 * s, pos + 3 * off, max_cutoff(h), 2, &Lst);
        if (rcode) break;
        double* dF = (double*)malloc(sizeof(double) * 3 * na);
        for (int k = 0; k < 3 * na; ++k) dF[k] = (Fall[3 * off + k] - f_tar[3 * off + k]) / (3.0 * ntot * L);
        double* gpart = (double*)calloc((size_t)na * npar, sizeof(double));
#pragma omp parallel
        {
            double* q = (double*)malloc(sizeof(double) * nd);
            double* x = (double*)malloc(sizeof(double) * nh);
            double* lam = (double*)malloc(sizeof(double) * nd);
            double* Jb = (double*)malloc(sizeof(double) * 3 * nd);
#pragma omp for schedule(dynamic, 8)
            for (int i = 0; i < na; ++i) {
                env E;
                env_alloc(h, &E, Lst.start[i + 1] - Lst.start[i], Lst.r + 3 * (size_t)Lst.start[i],
                          Zat ? Zat + off : NULL, i, Lst.j + Lst.start[i]);
                descriptor(h, &E, q);
                network(h, z, q, x, NULL);
                for (int v = 0; v < nd; ++v) lam[v] = 0.0;
                for (int a = 0; a < E.m; ++a) {
                    int j = Lst.j[Lst.start[i] + a];
                    descriptor_jacobian(h, &E, a, Jb);
                    double d[3] = {dF[3 * i] - dF[3 * j], dF[3 * i + 1] - dF[3 * j + 1], dF[3 * i + 2] - dF[3 * j + 2]};
                    for (int v = 0; v < nd; ++v) lam[v] += Jb[3 * v] * d[0] + Jb[3 * v + 1] * d[1] + Jb[3 * v + 2] * d[2];
                }
                double* g = gpart + (size_t)i * npar;
                for (int mu = 0; mu < nh; ++mu) {
                    double smu = 0.0;
                    for (int v = 0; v < nd; ++v) smu += w1[mu * nd + v] * lam[v];
                    double t = 1.0 - x[mu] * x[mu];
                    g[nh * nd + nh + mu] += t * smu;                            /* w2 */
                    g[nh * nd + mu] += 2.0 * w2[mu] * x[mu] * t * smu;          /* b1 */
                    for (int k = 0; k < nd; ++k)                                /* w1 */
                        g[mu * nd + k] += w2[mu] * t * lam[k] - 2.0 * w2[mu] * x[mu] * t * smu * q[k];
                }
                env_free(&E);
            }
            free(q);
            free(x);
            free(lam);
            free(Jb);
        }
        for (int i = 0; i < na; ++i)
            for (int k = 0; k < npar; ++k) grad[k] += gpart[(size_t)i * npar + k];
        free(gpart);
        free(dF);
        nlist_free(&Lst);
        off += na;
    }
    free(Fall);
    return rcode;
}

/* ------------------------------------------------------------------------ */
/* Separable natural evolution strategy, Eqs. 35-39.                         */
/* ------------------------------------------------------------------------ */
/*
 * Rank utilities (the paper defers the values to its reference; the standard
 * NES rank shaping is used): for rank k = 1..lambda (1 = lowest loss),
 * a_k = max(0, ln(lambda/2 + 1) - ln k), u_k = a_k / sum_j a_j - 1/lambda.
 */
void orc_snes_utilities(int npop, double* u)
{
    double sum = 0.0;
    for (int k = 1; k <= npop; ++k) {
        double a = log(npop / 2.0 + 1.0) - log((double)k);
        u[k - 1] = a > 0.0 ? a : 0.0;
        sum += u[k - 1];
    }
    for (int k = 0; k < npop; ++k) u[k] = u[k] / sum - 1.0 / npop;
}

/* learning rates of the paper: eta_m = 1, eta_s = (3 + ln N_par)/(5 sqrt N_par) */
double orc_snes_eta_s(int npar)
{
    return (3.0 + log((double)npar)) / (5.0 * sqrt((double)npar));
}

/*
 * One update of the search distribution from the population's losses and
 * the Gaussian draws r (npop x npar) that made z_k = m + s (.) r_k.
 * Members are ranked by ascending loss; equal losses keep index order.
 * m is updated with the pre-update s (Eq. 38), then s (Eq. 39).
 * order_out (npop) receives the member index at each rank (may be NULL).
 */
int orc_snes_update(int npar, int npop, const double* loss, const double* r, double* m, double* s, double eta_m,
                    double eta_s, int* order_out)
{
    if (npop < 2 || npar < 1) return ORC_ERR_ARG;
    int* order = (int*)malloc(sizeof(int) * npop);
    double* u = (double*)malloc(sizeof(double) * npop);
    for (int k = 0; k < npop; ++k) order[k] = k;
    /* stable insertion sort by loss */
    for (int a = 1; a < npop; ++a) {
        int key = order[a];
        int b = a - 1;
        while (b >= 0 && loss[order[b]] > loss[key]) {
            order[b + 1] = order[b];
            --b;
        }
        order[b + 1] = key;
    }
    orc_snes_utilities(npop, u);
    for (int p = 0; p < npar; ++p) {
        double gm = 0.0, gs = 0.0;
        for (int k = 0; k < npop; ++k) {
            double rv = r[(size_t)order[k] * npar + p];
            gm += u[k] * rv;
            gs += u[k] * (rv * rv - 1.0);
        }
        m[p] += eta_m * s[p] * gm;
        s[p] *= exp(0.5 * eta_s * gs);
    }
    if (order_out) memcpy(order_out, order, sizeof(int) * npop);
    free(order);
    free(u);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,        */
/* SC'11), written from its published definition, and Box-Muller normals.   */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t* ctr_in, const uint32_t* key_in, uint32_t* out)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k[2] = {key_in[0], key_in[1]};
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * c[0];
        uint64_t p1 = (uint64_t)M1 * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k[0];
        uint32_t n2 = hi0 ^ c[3] ^ k[1];
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k[0] += W0;
        k[1] += W1;
    }
    memcpy(out, c, sizeof(c));
}

/*
 * Standard normal draws for element e = 0..count-1 of stream (seed, gen):
 * block b = e / 4 uses counter {b, 0, gen, 0x4E4550u} and key {seed lo, seed hi};
 * with u_k = (w_k + 0.5) 2^-32, lanes 0/1 are sqrt(-2 ln u_0) cos/sin(2 pi u_1)
 * and lanes 2/3 the same with (u_2, u_3).
 */
void orc_gaussian(uint64_t seed, uint32_t gen, long count, double* out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (long e = 0; e < count; ++e) {
        uint32_t ctr[4] = {(uint32_t)(e / 4), 0u, gen, 0x4E4550u};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        int lane = (int)(e % 4);
        int pair = lane / 2;
        double u0 = ((double)w[2 * pair] + 0.5) * (1.0 / 4294967296.0);
        double u1 = ((double)w[2 * pair + 1] + 0.5) * (1.0 / 4294967296.0);
        double rad = sqrt(-2.0 * log(u0));
        out[e] = (lane % 2 == 0) ? rad * cos(2.0 * ORC_PI * u1) : rad * sin(2.0 * ORC_PI * u1);
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
