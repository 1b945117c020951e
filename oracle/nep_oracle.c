/*
 * nep_oracle.c -- plain, slow FP64 CPU oracle of the NEP energy / force / virial
 * evaluation used by NEP-CG and NEP-AACG (paper Sec. II.A and Sec. II.C).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed CPU
 * baseline load this library.  It shares no code, header, table or constant
 * generator with the CUDA library; it is written from the equations:
 *
 *   Eq. 1   E = sum_i U_i
 *   Eq. 2   U_i = sum_mu w1_mu tanh(sum_nu w0_{mu nu} q_nu - b0_mu) - b1
 *   Eq. 3   q_n   = sum_{j != i} g_n(r_ij)                    (radial)
 *   Eq. 4   q_nl  = sum_m (-1)^m A_nlm A_nl(-m)               (angular, 3-body)
 *   Eq. 5   A_nlm = sum_{j != i} g_n(r_ij) Y_lm(theta_ij, phi_ij)
 *   Eq. 6   g_n(r) = sum_{k=0}^{N_bas} c^{ij}_{nk} f_k(r)
 *   Eq. 7   f_k(r) = 1/2 [T_k(2 (r/r_c - 1)^2 - 1) + 1] f_c(r)
 *   Eq. 8   f_c(r) = 1/2 [1 + cos(pi r / r_c)] for r <= r_c, else 0
 *   Eq. 15  W_i = sum_{j != i} r_ij (x) dU_j/dr_ji,  r_ij = r_j - r_i
 *
 * Four- and five-body angular terms (Sec. II.A refers their definition to the
 * GPUMD paper, Fan et al., J. Chem. Phys. 157, 114801 (2022); read here as):
 *   q4_n = sum_{m1 m2 m3} (2 2 2; m1 m2 m3) A_n2m1 A_n2m2 A_n2m3   (Wigner 3j)
 *   q5_n = (q_n1)^2 = (sum_m (-1)^m A_n1m A_n1(-m))^2
 * the cubic invariant of the l = 2 moments and the quartic invariant of the l = 1
 * moments; each is the only rotational invariant of its degree, so these fix them
 * up to a constant factor, which the network weights absorb.
 *   Eq. 16  W = sum_i W_i
 *
 * Heat transport (the HNEMD runs of Sec. III.B follow Fan et al., Phys. Rev. B 99,
 * 064308 (2019), and the heat current of Fan et al., Phys. Rev. B 92, 094301 (2015)):
 *   J_pot = sum_i W_i v_i                        (W_i of Eq. 15 acting on v_i)
 *   J_kin = sum_i (1/2 m_i v_i^2 + U_i) v_i
 *   F_i^ext = F_e . W_i - (1/N) sum_j F_e . W_j  ((F_e . W)_b = sum_a Fe_a W_ab)
 * so that the driving forces add power F_e . J_pot and no net momentum.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - Y_lm are the complex orthonormal spherical harmonics with the Condon-Shortley
 *     phase; theta is the polar angle of r_ij, phi its azimuth.
 *   - A pair is a neighbour when r < r_c strictly (f_c and f_c' vanish at r_c).
 *   - j != i excludes only the zero-shift self image; periodic images of i count.
 *   - Descriptor order: q_0..q_{n_R-1}, then for l = 1..l_max, n = 0..n_A-1: q_nl,
 *     then q4_0..q4_{n_A-1} (when l_max^4b = 2), then q5_0..q5_{n_A-1} (when
 *     l_max^5b = 1).
 *   - Every parameter is per central type t_i; c is indexed (t_i, t_j).
 *   - Positions on periodic axes are wrapped to [0, L) before neighbours are
 *     searched: a position in [0, L) is kept, any other becomes x - L floor(x / L)
 *     (a result that rounds to L, or below 0, becomes 0).
 *
 * Forces are the analytic gradient F_k = -dE/dr_k.  The angular part of that
 * gradient is taken from the addition-theorem form of q_nl,
 *     q_nl = (2l+1)/(4 pi) sum_{a,b} g_n(r_a) g_n(r_b) P_l(u_a . u_b),
 * which is algebraically the same function as Eq. 4-5 but computed by a different
 * route, so that the finite-difference pin on forces cross-checks both.  The
 * four-body gradient likewise comes from a Cartesian form: with the traceless
 * tensor Q_n = sum_j g_n(r_j) (u_j u_j^T - I/3),
 *     q4_n = kappa tr(Q_n^3),  kappa = (2 2 2; 0 0 0) (5 / 4 pi)^(3/2) 9/2
 * (both sides are the cubic invariant of the l = 2 moments; one neighbour on the
 * z axis, where A_2m = g sqrt(5 / 4 pi) delta_m0 and tr(Q^3) = 2 g^3 / 9, fixes
 * kappa).  The five-body gradient is 2 q_n1 times that of q_n1.
 *
 * Units: Angstrom, eV, amu, fs.  All arithmetic is double precision.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* 1 eV / (Angstrom amu) expressed in Angstrom / fs^2 */
#define ORACLE_ACC 9.648533212e-3

/* ------------------------------------------------------------------------- */
/* Eq. 8 and its derivative                                                    */
/* ------------------------------------------------------------------------- */
double oracle_fc(double r, double rc)
{
    if (r > rc) return 0.0;
    return 0.5 * (1.0 + cos(M_PI * r / rc));
}

double oracle_dfc(double r, double rc)
{
    if (r > rc) return 0.0;
    return -0.5 * M_PI / rc * sin(M_PI * r / rc);
}

/* Chebyshev polynomial of the first kind by its closed form cos(k arccos x). */
double oracle_chebyshev(int k, double x)
{
    if (x > 1.0) x = 1.0;
    if (x < -1.0) x = -1.0;
    return cos(k * acos(x));
}

/* dT_k/dx = k sin(k arccos x) / sin(arccos x); at x = +-1 the limit (+-1)^(k+1) k^2. */
double oracle_dchebyshev(int k, double x)
{
    if (x >= 1.0) return (double)k * k;
    if (x <= -1.0) return ((k % 2) ? 1.0 : -1.0) * k * k;
    double th = acos(x);
    return k * sin(k * th) / sin(th);
}

/* Eq. 7: f_k(r) */
double oracle_fk(int k, double r, double rc)
{
    double s = r / rc - 1.0;
    double x = 2.0 * s * s - 1.0;
    return 0.5 * (oracle_chebyshev(k, x) + 1.0) * oracle_fc(r, rc);
}

/* d f_k / dr by the chain rule through x(r) = 2 (r/rc - 1)^2 - 1. */
double oracle_dfk(int k, double r, double rc)
{
    double s = r / rc - 1.0;
    double x = 2.0 * s * s - 1.0;
    double dxdr = 4.0 * s / rc;
    return 0.5 * oracle_dchebyshev(k, x) * dxdr * oracle_fc(r, rc)
         + 0.5 * (oracle_chebyshev(k, x) + 1.0) * oracle_dfc(r, rc);
}

/* Eq. 6: g_n(r) = sum_k c_k f_k(r), with K = N_bas + 1 coefficients c[0..K-1]. */
double oracle_gn(const double *c, int K, double r, double rc)
{
    double g = 0.0;
    for (int k = 0; k < K; ++k) g += c[k] * oracle_fk(k, r, rc);
    return g;
}

double oracle_dgn(const double *c, int K, double r, double rc)
{
    double g = 0.0;
    for (int k = 0; k < K; ++k) g += c[k] * oracle_dfk(k, r, rc);
    return g;
}

/* ------------------------------------------------------------------------- */
/* Legendre polynomials and spherical harmonics                                */
/* ------------------------------------------------------------------------- */
static double fact(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

static double binom(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    return fact(n) / (fact(k) * fact(n - k));
}

/* m-th derivative of P_l at x, from the explicit sum
 *   P_l(x) = 2^-l sum_{k=0}^{floor(l/2)} (-1)^k C(l,k) C(2l-2k,l) x^(l-2k). */
static double legendre_dm(int l, int m, double x)
{
    double s = 0.0;
    for (int k = 0; 2 * k <= l; ++k) {
        int p = l - 2 * k;
        if (p < m) continue;
        double term = ((k % 2) ? -1.0 : 1.0) * binom(l, k) * binom(2 * l - 2 * k, l)
                    * fact(p) / fact(p - m) * pow(x, p - m);
        s += term;
    }
    return s / pow(2.0, l);
}

double oracle_legendre(int l, double x) { return legendre_dm(l, 0, x); }
double oracle_dlegendre(int l, double x) { return legendre_dm(l, 1, x); }

/* Associated Legendre function P_l^m(x), 0 <= m <= l, Condon-Shortley phase:
 *   P_l^m(x) = (-1)^m (1 - x^2)^(m/2) d^m P_l / dx^m. */
double oracle_assoc_legendre(int l, int m, double x)
{
    double w = 1.0 - x * x;
    if (w < 0.0) w = 0.0;
    return ((m % 2) ? -1.0 : 1.0) * pow(w, 0.5 * m) * legendre_dm(l, m, x);
}

/* Complex orthonormal spherical harmonic Y_lm(theta, phi). */
void oracle_ylm(int l, int m, double theta, double phi, double *re, double *im)
{
    int am = m < 0 ? -m : m;
    double norm = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * fact(l - am) / fact(l + am));
    double p = norm * oracle_assoc_legendre(l, am, cos(theta));
    double yr = p * cos(am * phi), yi = p * sin(am * phi);
    if (m < 0) { /* Y_{l,-m} = (-1)^m conj(Y_lm) */
        double sg = (am % 2) ? -1.0 : 1.0;
        yr = sg * yr;
        yi = -sg * yi;
    }
    *re = yr;
    *im = yi;
}

/* Wigner 3j symbol (j1 j2 j3; m1 m2 m3) for integer arguments, by Racah's
 * single-sum formula. */
double oracle_wigner3j(int j1, int j2, int j3, int m1, int m2, int m3)
{
    if (m1 + m2 + m3 != 0) return 0.0;
    if (j3 < abs(j1 - j2) || j3 > j1 + j2) return 0.0;
    if (abs(m1) > j1 || abs(m2) > j2 || abs(m3) > j3) return 0.0;
    double tri = fact(j1 + j2 - j3) * fact(j1 - j2 + j3) * fact(-j1 + j2 + j3) / fact(j1 + j2 + j3 + 1);
    double pre = sqrt(tri * fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) * fact(j2 - m2) * fact(j3 + m3) *
                      fact(j3 - m3));
    double s = 0.0;
    for (int k = 0; k <= j1 + j2 + j3; ++k) {
        int a1 = j3 - j2 + k + m1, a2 = j3 - j1 + k - m2, a3 = j1 + j2 - j3 - k, a4 = j1 - k - m1,
            a5 = j2 - k + m2;
        if (a1 < 0 || a2 < 0 || a3 < 0 || a4 < 0 || a5 < 0) continue;
        s += ((k % 2) ? -1.0 : 1.0) / (fact(k) * fact(a1) * fact(a2) * fact(a3) * fact(a4) * fact(a5));
    }
    int ph = j1 - j2 - m3;
    return ((ph % 2 + 2) % 2 ? -1.0 : 1.0) * pre * s;
}

/* ------------------------------------------------------------------------- */
/* Model                                                                       */
/* ------------------------------------------------------------------------- */
typedef struct {
    int T, nR, nA, KR, KA, L, L4, L5, H;
    const double *rcR, *rcA;           /* [T][T] */
    const double *cR, *cA;             /* [T][T][nR][KR], [T][T][nA][KA] */
    const double *w0, *b0, *w1, *b1;   /* [T][H][Ndes], [T][H], [T][H], [T] */
} omodel;

static int ndes(const omodel *m) { return m->nR + m->nA * (m->L + (m->L4 > 0) + (m->L5 > 0)); }
/* indices of q4_n and q5_n in the descriptor vector */
static int q4_index(const omodel *m, int n) { return m->nR + m->nA * m->L + n; }
static int q5_index(const omodel *m, int n) { return m->nR + m->nA * (m->L + (m->L4 > 0)) + n; }
static const double *coefR(const omodel *m, int ti, int tj, int n) { return m->cR + (((size_t)ti * m->T + tj) * m->nR + n) * m->KR; }
static const double *coefA(const omodel *m, int ti, int tj, int n) { return m->cA + (((size_t)ti * m->T + tj) * m->nA + n) * m->KA; }

/* ------------------------------------------------------------------------- */
/* Neighbours                                                                  */
/* ------------------------------------------------------------------------- */
typedef struct {
    int j;
    int s[3];       /* image shift in box lengths */
    int inR, inA;   /* radial / angular membership */
} opair;

typedef struct {
    int n;
    int *start;     /* [n+1] CSR offsets */
    opair *p;
} olist;

static double wrap1(double x, double L)
{
    if (x >= 0.0 && x < L) return x;  /* inside the box: kept */
    double w = x - L * floor(x / L);
    if (w >= L) w = 0.0;
    if (w < 0.0) w = 0.0;
    return w;
}

void oracle_wrap(int n, const double *pos, const double box[3], const int pbc[3], double *out)
{
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < n; ++i)
            out[(size_t)a * n + i] = pbc[a] ? wrap1(pos[(size_t)a * n + i], box[a]) : pos[(size_t)a * n + i];
}

static void pair_vec(const double *w, int n, const double box[3], int i, const opair *p, double d[3])
{
    for (int a = 0; a < 3; ++a)
        d[a] = (w[(size_t)a * n + p->j] + p->s[a] * box[a]) - w[(size_t)a * n + i];
}

static int cmp_pair(const void *x, const void *y)
{
    const opair *a = (const opair *)x, *b = (const opair *)y;
    if (a->j != b->j) return a->j < b->j ? -1 : 1;
    for (int k = 0; k < 3; ++k)
        if (a->s[k] != b->s[k]) return a->s[k] < b->s[k] ? -1 : 1;
    return 0;
}

/* Classify candidate (i, j, shift); returns 1 if it is a neighbour. */
static int classify(const omodel *m, const double *w, int n, const int *types, const double box[3],
                    int i, opair *p)
{
    if (p->j == i && p->s[0] == 0 && p->s[1] == 0 && p->s[2] == 0) return 0;
    double d[3];
    pair_vec(w, n, box, i, p, d);
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    int ti = types[i], tj = types[p->j];
    double rR = m->rcR[ti * m->T + tj], rA = m->rcA[ti * m->T + tj];
    p->inR = r2 < rR * rR;
    p->inA = r2 < rA * rA;
    return p->inR || p->inA;
}

/* Brute force: every j, every image shift with |s_a| <= ceil(rc_max / L_a) + 1 on
 * periodic axes. Two passes (count, fill), then each bead's list is sorted. */
static int build_brute(const omodel *m, int n, const int *types, const double *w, const double box[3],
                       const int pbc[3], olist *out)
{
    double rcm = 0.0;
    for (int a = 0; a < m->T * m->T; ++a) {
        if (m->rcR[a] > rcm) rcm = m->rcR[a];
        if (m->rcA[a] > rcm) rcm = m->rcA[a];
    }
    int S[3];
    for (int a = 0; a < 3; ++a) S[a] = pbc[a] ? (int)ceil(rcm / box[a]) + 1 : 0;
    int *cnt = (int *)calloc((size_t)n + 1, sizeof(int));
    if (!cnt) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        int c = 0;
        opair p;
        for (int j = 0; j < n; ++j)
            for (p.s[0] = -S[0]; p.s[0] <= S[0]; ++p.s[0])
                for (p.s[1] = -S[1]; p.s[1] <= S[1]; ++p.s[1])
                    for (p.s[2] = -S[2]; p.s[2] <= S[2]; ++p.s[2]) {
                        p.j = j;
                        c += classify(m, w, n, types, box, i, &p);
                    }
        cnt[i] = c;
    }
    out->n = n;
    out->start = (int *)malloc(((size_t)n + 1) * sizeof(int));
    out->start[0] = 0;
    for (int i = 0; i < n; ++i) out->start[i + 1] = out->start[i] + cnt[i];
    out->p = (opair *)malloc((size_t)out->start[n] * sizeof(opair) + 1);
    free(cnt);
    if (!out->p) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        int c = out->start[i];
        opair p;
        for (int j = 0; j < n; ++j)
            for (p.s[0] = -S[0]; p.s[0] <= S[0]; ++p.s[0])
                for (p.s[1] = -S[1]; p.s[1] <= S[1]; ++p.s[1])
                    for (p.s[2] = -S[2]; p.s[2] <= S[2]; ++p.s[2]) {
                        p.j = j;
                        if (classify(m, w, n, types, box, i, &p)) out->p[c++] = p;
                    }
        qsort(out->p + out->start[i], (size_t)(out->start[i + 1] - out->start[i]), sizeof(opair), cmp_pair);
    }
    return 0;
}

/* Cell list: periodic axes need at least 3 cells of side >= rc_max (otherwise the
 * caller uses brute force); open axes are binned over the positions' extent. */
static int build_cells(const omodel *m, int n, const int *types, const double *w, const double box[3],
                       const int pbc[3], olist *out)
{
    double rcm = 0.0;
    for (int a = 0; a < m->T * m->T; ++a) {
        if (m->rcR[a] > rcm) rcm = m->rcR[a];
        if (m->rcA[a] > rcm) rcm = m->rcA[a];
    }
    int nc[3];
    double lo[3], len[3];
    for (int a = 0; a < 3; ++a) {
        if (pbc[a]) {
            lo[a] = 0.0;
            nc[a] = (int)floor(box[a] / rcm);
            if (nc[a] < 3) return 1; /* not applicable */
            len[a] = box[a] / nc[a];
        } else {
            double mn = 1e300, mx = -1e300;
            for (int i = 0; i < n; ++i) {
                double x = w[(size_t)a * n + i];
                if (x < mn) mn = x;
                if (x > mx) mx = x;
            }
            lo[a] = mn;
            nc[a] = (int)floor((mx - mn) / rcm);
            if (nc[a] < 1) nc[a] = 1;
            len[a] = (mx - mn) / nc[a];
            if (len[a] < rcm) len[a] = rcm;
        }
    }
    size_t ncell = (size_t)nc[0] * nc[1] * nc[2];
    int *cell = (int *)malloc((size_t)n * sizeof(int));
    int *head = (int *)calloc(ncell + 1, sizeof(int));
    int *item = (int *)malloc((size_t)n * sizeof(int));
    int *fill = (int *)calloc(ncell, sizeof(int));
    int *cnt = (int *)calloc((size_t)n + 1, sizeof(int));
    if (!cell || !head || !item || !fill || !cnt) return -1;
    for (int i = 0; i < n; ++i) {
        int c3[3];
        for (int a = 0; a < 3; ++a) {
            int c = (int)floor((w[(size_t)a * n + i] - lo[a]) / len[a]);
            if (c < 0) c = 0;
            if (c >= nc[a]) c = nc[a] - 1;
            c3[a] = c;
        }
        cell[i] = (c3[2] * nc[1] + c3[1]) * nc[0] + c3[0];
        head[cell[i] + 1]++;
    }
    for (size_t c = 0; c < ncell; ++c) head[c + 1] += head[c];
    for (int i = 0; i < n; ++i) item[head[cell[i]] + fill[cell[i]]++] = i;

    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            out->n = n;
            out->start = (int *)malloc(((size_t)n + 1) * sizeof(int));
            out->start[0] = 0;
            for (int i = 0; i < n; ++i) out->start[i + 1] = out->start[i] + cnt[i];
            out->p = (opair *)malloc((size_t)out->start[n] * sizeof(opair) + 1);
        }
#pragma omp parallel for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            int ci[3] = {cell[i] % nc[0], (cell[i] / nc[0]) % nc[1], cell[i] / (nc[0] * nc[1])};
            int c = 0, base = pass ? out->start[i] : 0;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int dd[3] = {dx, dy, dz}, cc[3], sh[3], ok = 1;
                        for (int a = 0; a < 3; ++a) {
                            int v = ci[a] + dd[a];
                            sh[a] = 0;
                            if (pbc[a]) {
                                if (v < 0) { v += nc[a]; sh[a] = -1; }
                                if (v >= nc[a]) { v -= nc[a]; sh[a] = 1; }
                            } else if (v < 0 || v >= nc[a]) ok = 0;
                            cc[a] = v;
                        }
                        if (!ok) continue;
                        int cid = (cc[2] * nc[1] + cc[1]) * nc[0] + cc[0];
                        for (int q = head[cid]; q < head[cid + 1]; ++q) {
                            opair p;
                            p.j = item[q];
                            p.s[0] = sh[0]; p.s[1] = sh[1]; p.s[2] = sh[2];
                            if (classify(m, w, n, types, box, i, &p)) {
                                if (pass) out->p[base + c] = p;
                                ++c;
                            }
                        }
                    }
            if (pass == 0) cnt[i] = c;
            else qsort(out->p + out->start[i], (size_t)c, sizeof(opair), cmp_pair);
        }
    }
    free(cell); free(head); free(item); free(fill); free(cnt);
    return 0;
}

static void free_list(olist *l)
{
    free(l->start);
    free(l->p);
    l->start = NULL;
    l->p = NULL;
}

static int build_list(const omodel *m, int n, const int *types, const double *w, const double box[3],
                      const int pbc[3], int use_cells, olist *out)
{
    if (use_cells) {
        int rc = build_cells(m, n, types, w, box, pbc, out);
        if (rc <= 0) return rc;
    }
    return build_brute(m, n, types, w, box, pbc, out);
}

/* Neighbour export: pairs (i, j, sx, sy, sz, inR, inA) in the canonical order
 * (by i, then j, then shift).  Returns the number of pairs, or -needed if
 * max_pairs is too small, or -1 on allocation failure (needed >= 1 always). */
long oracle_neighbors(int T, const double *rcR, const double *rcA, int n, const int *types,
                      const double *pos, const double box[3], const int pbc[3], int use_cells,
                      long max_pairs, int *out /* [max_pairs][7] */)
{
    omodel m;
    memset(&m, 0, sizeof m);
    m.T = T; m.rcR = rcR; m.rcA = rcA;
    double *w = (double *)malloc((size_t)3 * n * sizeof(double) + 8);
    oracle_wrap(n, pos, box, pbc, w);
    olist l;
    if (build_list(&m, n, types, w, box, pbc, use_cells, &l)) { free(w); return -1; }
    long np = l.start[n];
    if (np > max_pairs) { free_list(&l); free(w); return -(np + 1); }
    for (int i = 0; i < n; ++i)
        for (int q = l.start[i]; q < l.start[i + 1]; ++q) {
            int *o = out + (size_t)q * 7;
            o[0] = i; o[1] = l.p[q].j;
            o[2] = l.p[q].s[0]; o[3] = l.p[q].s[1]; o[4] = l.p[q].s[2];
            o[5] = l.p[q].inR; o[6] = l.p[q].inA;
        }
    free_list(&l);
    free(w);
    return np;
}

/* ------------------------------------------------------------------------- */
/* Descriptors, network, gradients                                             */
/* ------------------------------------------------------------------------- */

/* Eq. 3-5 for bead i: radial q_n and angular q_nl via complex Y_lm (the
 * definition).  q[0..ndes) in the documented order. */
static void descriptor_ylm(const omodel *m, int n, const int *types, const double *w, const double box[3],
                           const olist *l, int i, double *q)
{
    int ti = types[i];
    for (int k = 0; k < ndes(m); ++k) q[k] = 0.0;
    /* A[n][l][m+l], complex, l <= 4 (l <= 2 is also needed by the 4-body term) */
    double Ar[16][5][9], Ai[16][5][9];
    int lacc = m->L > 2 ? m->L : 2;
    memset(Ar, 0, sizeof Ar);
    memset(Ai, 0, sizeof Ai);
    for (int a = l->start[i]; a < l->start[i + 1]; ++a) {
        const opair *p = &l->p[a];
        int tj = types[p->j];
        double d[3];
        pair_vec(w, n, box, i, p, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (p->inR) {
            double rc = m->rcR[ti * m->T + tj];
            for (int nn = 0; nn < m->nR; ++nn) q[nn] += oracle_gn(coefR(m, ti, tj, nn), m->KR, r, rc);
        }
        if (p->inA) {
            double rc = m->rcA[ti * m->T + tj];
            double theta = acos(d[2] / r), phi = atan2(d[1], d[0]);
            for (int nn = 0; nn < m->nA; ++nn) {
                double g = oracle_gn(coefA(m, ti, tj, nn), m->KA, r, rc);
                for (int ll = 1; ll <= lacc; ++ll)
                    for (int mm = -ll; mm <= ll; ++mm) {
                        double yr, yi;
                        oracle_ylm(ll, mm, theta, phi, &yr, &yi);
                        Ar[nn][ll][mm + ll] += g * yr;
                        Ai[nn][ll][mm + ll] += g * yi;
                    }
            }
        }
    }
    for (int ll = 1; ll <= m->L; ++ll)
        for (int nn = 0; nn < m->nA; ++nn) {
            double s = 0.0;
            for (int mm = -ll; mm <= ll; ++mm) {
                /* (-1)^m A_nlm A_nl(-m), real part (the imaginary part cancels) */
                double ar = Ar[nn][ll][mm + ll], ai = Ai[nn][ll][mm + ll];
                double br = Ar[nn][ll][-mm + ll], bi = Ai[nn][ll][-mm + ll];
                double sg = (mm % 2) ? -1.0 : 1.0;
                s += sg * (ar * br - ai * bi);
            }
            q[m->nR + (ll - 1) * m->nA + nn] = s;
        }
    /* four-body: sum over m1 + m2 + m3 = 0 of the 3j-weighted triple product (real
     * part; the imaginary part cancels because A_l(-m) = (-1)^m conj(A_lm)) */
    if (m->L4)
        for (int nn = 0; nn < m->nA; ++nn) {
            double s = 0.0;
            for (int m1 = -2; m1 <= 2; ++m1)
                for (int m2 = -2; m2 <= 2; ++m2) {
                    int m3 = -m1 - m2;
                    if (m3 < -2 || m3 > 2) continue;
                    double c = oracle_wigner3j(2, 2, 2, m1, m2, m3);
                    double ar = Ar[nn][2][m1 + 2], ai = Ai[nn][2][m1 + 2];
                    double br = Ar[nn][2][m2 + 2], bi = Ai[nn][2][m2 + 2];
                    double cr = Ar[nn][2][m3 + 2], ci = Ai[nn][2][m3 + 2];
                    double pr = ar * br - ai * bi, pi = ar * bi + ai * br;
                    s += c * (pr * cr - pi * ci);
                }
            q[q4_index(m, nn)] = s;
        }
    /* five-body: the square of the l = 1 pair coupling */
    if (m->L5)
        for (int nn = 0; nn < m->nA; ++nn) {
            double s = 0.0;
            for (int mm = -1; mm <= 1; ++mm) {
                double ar = Ar[nn][1][mm + 1], ai = Ai[nn][1][mm + 1];
                double br = Ar[nn][1][-mm + 1], bi = Ai[nn][1][-mm + 1];
                s += ((mm % 2) ? -1.0 : 1.0) * (ar * br - ai * bi);
            }
            q[q5_index(m, nn)] = s * s;
        }
}

/* Angular q_nl by the addition theorem (Legendre double sum over the angular
 * neighbours, j = k terms included). */
static void descriptor_legendre(const omodel *m, int n, const int *types, const double *w, const double box[3],
                                const olist *l, int i, double *q)
{
    int ti = types[i];
    for (int ll = 1; ll <= m->L; ++ll)
        for (int nn = 0; nn < m->nA; ++nn) q[m->nR + (ll - 1) * m->nA + nn] = 0.0;
    for (int a = l->start[i]; a < l->start[i + 1]; ++a) {
        const opair *pa = &l->p[a];
        if (!pa->inA) continue;
        double da[3];
        pair_vec(w, n, box, i, pa, da);
        double ra = sqrt(da[0] * da[0] + da[1] * da[1] + da[2] * da[2]);
        int ta = types[pa->j];
        for (int b = l->start[i]; b < l->start[i + 1]; ++b) {
            const opair *pb = &l->p[b];
            if (!pb->inA) continue;
            double db[3];
            pair_vec(w, n, box, i, pb, db);
            double rb = sqrt(db[0] * db[0] + db[1] * db[1] + db[2] * db[2]);
            int tb = types[pb->j];
            double c = (da[0] * db[0] + da[1] * db[1] + da[2] * db[2]) / (ra * rb);
            for (int nn = 0; nn < m->nA; ++nn) {
                double ga = oracle_gn(coefA(m, ti, ta, nn), m->KA, ra, m->rcA[ti * m->T + ta]);
                double gb = oracle_gn(coefA(m, ti, tb, nn), m->KA, rb, m->rcA[ti * m->T + tb]);
                for (int ll = 1; ll <= m->L; ++ll)
                    q[m->nR + (ll - 1) * m->nA + nn] += (2.0 * ll + 1.0) / (4.0 * M_PI) * ga * gb * oracle_legendre(ll, c);
            }
        }
    }
}

/* Eq. 2 and its gradient dU/dq. */
static double network(const omodel *m, int t, const double *q, double *dUdq)
{
    int D = ndes(m);
    const double *w0 = m->w0 + (size_t)t * m->H * D;
    const double *b0 = m->b0 + (size_t)t * m->H;
    const double *w1 = m->w1 + (size_t)t * m->H;
    double U = -m->b1[t];
    if (dUdq)
        for (int v = 0; v < D; ++v) dUdq[v] = 0.0;
    for (int mu = 0; mu < m->H; ++mu) {
        double x = -b0[mu];
        for (int v = 0; v < D; ++v) x += w0[mu * D + v] * q[v];
        double h = tanh(x);
        U += w1[mu] * h;
        if (dUdq)
            for (int v = 0; v < D; ++v) dUdq[v] += w1[mu] * (1.0 - h * h) * w0[mu * D + v];
    }
    return U;
}

/* dU_i/d(r_ij) for the pair a of bead i, given bead i's descriptors q and dU_i/dq
 * (grad). */
static void pair_gradient(const omodel *m, int n, const int *types, const double *w, const double box[3],
                          const olist *l, int i, int a, const double *q, const double *grad, double out[3])
{
    int ti = types[i];
    const opair *pa = &l->p[a];
    int ta = types[pa->j];
    double da[3];
    pair_vec(w, n, box, i, pa, da);
    double ra = sqrt(da[0] * da[0] + da[1] * da[1] + da[2] * da[2]);
    double ua[3] = {da[0] / ra, da[1] / ra, da[2] / ra};
    out[0] = out[1] = out[2] = 0.0;
    if (pa->inR) {
        double rc = m->rcR[ti * m->T + ta], s = 0.0;
        for (int nn = 0; nn < m->nR; ++nn) s += grad[nn] * oracle_dgn(coefR(m, ti, ta, nn), m->KR, ra, rc);
        for (int k = 0; k < 3; ++k) out[k] += s * ua[k];
    }
    if (!pa->inA) return;
    /* d q_nl / d r_a = (2l+1)/(4 pi) * 2 sum_b [ g'(a) g(b) P_l(c) u_a
     *                                           + g(a) g(b) P_l'(c) (u_b - c u_a)/r_a ] */
    double rcA = m->rcA[ti * m->T + ta];
    double gA[16], dgA[16];
    for (int nn = 0; nn < m->nA; ++nn) {
        gA[nn] = oracle_gn(coefA(m, ti, ta, nn), m->KA, ra, rcA);
        dgA[nn] = oracle_dgn(coefA(m, ti, ta, nn), m->KA, ra, rcA);
    }
    for (int b = l->start[i]; b < l->start[i + 1]; ++b) {
        const opair *pb = &l->p[b];
        if (!pb->inA) continue;
        int tb = types[pb->j];
        double db[3];
        pair_vec(w, n, box, i, pb, db);
        double rb = sqrt(db[0] * db[0] + db[1] * db[1] + db[2] * db[2]);
        double ub[3] = {db[0] / rb, db[1] / rb, db[2] / rb};
        double c = ua[0] * ub[0] + ua[1] * ub[1] + ua[2] * ub[2];
        double t[3] = {(ub[0] - c * ua[0]) / ra, (ub[1] - c * ua[1]) / ra, (ub[2] - c * ua[2]) / ra};
        for (int nn = 0; nn < m->nA; ++nn) {
            double ga = gA[nn], dga = dgA[nn];
            double gb = oracle_gn(coefA(m, ti, tb, nn), m->KA, rb, m->rcA[ti * m->T + tb]);
            for (int ll = 1; ll <= m->L; ++ll) {
                double dq = grad[m->nR + (ll - 1) * m->nA + nn];
                if (ll == 1 && m->L5) dq += 2.0 * q[m->nR + nn] * grad[q5_index(m, nn)];  /* q5 = q_n1^2 */
                double G = dq * 2.0 * (2.0 * ll + 1.0) / (4.0 * M_PI);
                double P = oracle_legendre(ll, c), dP = oracle_dlegendre(ll, c);
                for (int k = 0; k < 3; ++k) out[k] += G * (dga * gb * P * ua[k] + ga * gb * dP * t[k]);
            }
        }
    }
    if (!m->L4) return;
    /* four-body: d q4 / d r_a = 3 kappa tr(Q^2 dQ/dr_a), Q = sum_b g(r_b) (u_b u_b^T - I/3) */
    const double kappa = oracle_wigner3j(2, 2, 2, 0, 0, 0) * pow(5.0 / (4.0 * M_PI), 1.5) * 4.5;
    for (int nn = 0; nn < m->nA; ++nn) {
        double Q[3][3] = {{0}};
        for (int b = l->start[i]; b < l->start[i + 1]; ++b) {
            const opair *pb = &l->p[b];
            if (!pb->inA) continue;
            int tb = types[pb->j];
            double db[3];
            pair_vec(w, n, box, i, pb, db);
            double rb = sqrt(db[0] * db[0] + db[1] * db[1] + db[2] * db[2]);
            double gb = oracle_gn(coefA(m, ti, tb, nn), m->KA, rb, m->rcA[ti * m->T + tb]);
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y) Q[x][y] += gb * (db[x] * db[y] / (rb * rb) - (x == y ? 1.0 / 3.0 : 0.0));
        }
        double Q2[3][3], trQ2 = 0.0;
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) {
                Q2[x][y] = Q[x][0] * Q[0][y] + Q[x][1] * Q[1][y] + Q[x][2] * Q[2][y];
                if (x == y) trQ2 += Q2[x][y];
            }
        double Q2u[3], uQ2u = 0.0;
        for (int x = 0; x < 3; ++x) {
            Q2u[x] = Q2[x][0] * ua[0] + Q2[x][1] * ua[1] + Q2[x][2] * ua[2];
            uQ2u += ua[x] * Q2u[x];
        }
        double G = 3.0 * kappa * grad[q4_index(m, nn)];
        for (int k = 0; k < 3; ++k)
            out[k] += G * (dgA[nn] * (uQ2u - trQ2 / 3.0) * ua[k] + 2.0 * gA[nn] * (Q2u[k] - uQ2u * ua[k]) / ra);
    }
}

/* index in j's list of the pair that points back at (i, -s); -1 if absent */
static int reverse_pair(const olist *l, int i, const opair *p)
{
    for (int b = l->start[p->j]; b < l->start[p->j + 1]; ++b) {
        const opair *q = &l->p[b];
        if (q->j == i && q->s[0] == -p->s[0] && q->s[1] == -p->s[1] && q->s[2] == -p->s[2]) return b;
    }
    return -1;
}

/*
 * Energy, forces and virials.
 *   sample == NULL: every bead; energy_total / virial_total are filled.
 *   sample != NULL: only the listed beads' U, F, W (and q if requested) are
 *                   written at their own index; totals are left untouched.
 * Outputs: U [n], F SoA [3][n], W [9][n] (row-major alpha,beta: W[3a+b][i]),
 *          q [n][ndes] (optional), angular route: 0 = Y_lm (Eq. 4-5),
 *          1 = Legendre double sum.
 * Returns 0, or -1 on allocation failure / missing reverse pair.
 */
int oracle_compute(int T, int nR, int nA, int KR, int KA, int L, int L4, int L5, int H,
                   const double *rcR, const double *rcA, const double *cR, const double *cA,
                   const double *w0, const double *b0, const double *w1, const double *b1,
                   int n, const int *types, const double *pos, const double box[3], const int pbc[3],
                   int use_cells, const int *sample, int n_sample, int q_route,
                   double *energy_total, double *virial_total, double *U, double *F, double *W,
                   double *q_out)
{
    omodel m = {T, nR, nA, KR, KA, L, L4, L5, H, rcR, rcA, cR, cA, w0, b0, w1, b1};
    if (L < 1 || L > 4 || nA > 16 || nR > 16 || (L4 != 0 && L4 != 2) || (L5 != 0 && L5 != 1)) return -1;
    int D = ndes(&m);
    double *w = (double *)malloc((size_t)3 * n * sizeof(double) + 8);
    oracle_wrap(n, pos, box, pbc, w);
    olist l;
    if (build_list(&m, n, types, w, box, pbc, use_cells, &l)) { free(w); return -1; }

    /* beads whose network gradient is needed: the sample and their neighbours */
    char *need = (char *)calloc((size_t)n, 1);
    char *is_sample = (char *)calloc((size_t)n, 1);
    if (sample) {
        for (int s = 0; s < n_sample; ++s) {
            int i = sample[s];
            is_sample[i] = need[i] = 1;
            for (int a = l.start[i]; a < l.start[i + 1]; ++a) need[l.p[a].j] = 1;
        }
    } else {
        memset(need, 1, (size_t)n);
        memset(is_sample, 1, (size_t)n);
    }
    double *grad = (double *)calloc((size_t)n * D, sizeof(double));
    double *qall = (double *)calloc((size_t)n * D, sizeof(double));
    double *Ui = (double *)calloc((size_t)n, sizeof(double));
    double *pg = (double *)calloc((size_t)l.start[n] * 3 + 3, sizeof(double));
    int err = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        if (!need[i]) continue;
        double *q = qall + (size_t)i * D;
        descriptor_ylm(&m, n, types, w, box, &l, i, q);
        if (q_route == 1) descriptor_legendre(&m, n, types, w, box, &l, i, q);
        Ui[i] = network(&m, types[i], q, grad + (size_t)i * D);
        if (q_out && is_sample[i])
            for (int k = 0; k < D; ++k) q_out[(size_t)i * D + k] = q[k];
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        if (!need[i]) continue;
        for (int a = l.start[i]; a < l.start[i + 1]; ++a)
            pair_gradient(&m, n, types, w, box, &l, i, a, qall + (size_t)i * D, grad + (size_t)i * D,
                          pg + (size_t)a * 3);
    }
    /* F_i = sum_j (dU_i/dr_ij - dU_j/dr_ji);  W_i = sum_j r_ij (x) dU_j/dr_ji  (Eq. 15) */
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        if (!is_sample[i]) continue;
        double f[3] = {0, 0, 0}, v[9] = {0};
        for (int a = l.start[i]; a < l.start[i + 1]; ++a) {
            const opair *p = &l.p[a];
            int b = reverse_pair(&l, i, p);
            if (b < 0) { err = 1; continue; }
            double d[3];
            pair_vec(w, n, box, i, p, d);
            const double *gij = pg + (size_t)a * 3, *gji = pg + (size_t)b * 3;
            for (int k = 0; k < 3; ++k) f[k] += gij[k] - gji[k];
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y) v[3 * x + y] += d[x] * gji[y];
        }
        if (U) U[i] = Ui[i];
        if (F)
            for (int k = 0; k < 3; ++k) F[(size_t)k * n + i] = f[k];
        if (W)
            for (int k = 0; k < 9; ++k) W[(size_t)k * n + i] = v[k];
    }
    if (!sample && energy_total) {
        double e = 0.0;
        for (int i = 0; i < n; ++i) e += Ui[i];
        *energy_total = e;
    }
    if (!sample && virial_total && W) {
        for (int k = 0; k < 9; ++k) {
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += W[(size_t)k * n + i];
            virial_total[k] = s;
        }
    }
    free(grad); free(qall); free(Ui); free(pg); free(need); free(is_sample);
    free_list(&l);
    free(w);
    return err ? -1 : 0;
}

/*
 * HNEMD driving force (Fan et al. 2019): F_i += F_e . W_i - (1/N) sum_j F_e . W_j,
 * with (F_e . W_i)_b = sum_a Fe_a W_i[a][b] and W_i the per-particle virial of
 * Eq. 15 (SoA [9][n], row-major 3x3).  force SoA [3][n], updated in place.
 */
void oracle_hnemd_force(int n, const double fe[3], const double *W, double *force)
{
    double mean[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < n; ++i)
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) mean[b] += fe[a] * W[(size_t)(3 * a + b) * n + i];
    for (int b = 0; b < 3; ++b) mean[b] /= n;
    for (int i = 0; i < n; ++i)
        for (int b = 0; b < 3; ++b) {
            double f = 0.0;
            for (int a = 0; a < 3; ++a) f += fe[a] * W[(size_t)(3 * a + b) * n + i];
            force[(size_t)b * n + i] += f - mean[b];
        }
}

/*
 * Heat current of a many-body potential (Fan et al. 2015), in eV Angstrom / fs:
 *   J_pot[a] = sum_i sum_b W_i[a][b] v_i[b]
 *   J_kin[a] = sum_i (1/2 m_i |v_i|^2 + U_i) v_i[a]
 * vel SoA [3][n] (Angstrom/fs), U [n] (eV), W SoA [9][n]; out[6] = J_pot, J_kin.
 */
void oracle_heat_current(int n, const int *types, const double *masses, const double *vel, const double *U,
                         const double *W, double out[6])
{
    for (int k = 0; k < 6; ++k) out[k] = 0.0;
    for (int i = 0; i < n; ++i) {
        double v[3], v2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            v[a] = vel[(size_t)a * n + i];
            v2 += v[a] * v[a];
        }
        double Ei = 0.5 * masses[types[i]] * v2 / ORACLE_ACC + U[i];
        for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) out[a] += W[(size_t)(3 * a + b) * n + i] * v[b];
            out[3 + a] += Ei * v[a];
        }
    }
}

/*
 * Velocity-Verlet (the integrator of the MD step):
 *   v += dt/2 F/m;  r += dt v;  wrap periodic axes;  F = F(r);  v += dt/2 F/m.
 * With noise != NULL every step ends with stochastic velocity rescaling (Bussi,
 * Donadio and Parrinello 2007): the kinetic energy K is resampled as
 *   K' = c K + (1 - c) (Kbar / N_f) (R1^2 + S) + 2 R1 sqrt(c (1 - c) K Kbar / N_f)
 * with c = exp(-dt / tau), N_f = 3n - 3, Kbar = N_f k_B T / 2 and the step's
 * noise (R1, S), and all velocities are scaled by sqrt(K' / K).
 * With fe != NULL the HNEMD driving force of F_e = fe[3] (1/Angstrom) is added to
 * the force after every evaluation (oracle_hnemd_force), before the second kick.
 * pos, vel, force: SoA [3][n], in/out; force must hold the total force at pos on
 * entry (with the driving force when fe != NULL).
 * masses: per type (amu).  thermo (optional) [n_steps][2]: potential energy and
 * kinetic energy after each step.  heat (optional) [n_steps][6]: J_pot and J_kin
 * (eV Angstrom / fs) after each step, thermostat included.
 */
int oracle_md(int T, int nR, int nA, int KR, int KA, int L, int L4, int L5, int H,
              const double *rcR, const double *rcA, const double *cR, const double *cA,
              const double *w0, const double *b0, const double *w1, const double *b1,
              int n, const int *types, double *pos, double *vel, double *force, const double *masses,
              const double box[3], const int pbc[3], int use_cells, int n_steps, double dt, double *thermo,
              double temperature, double tau, const double *noise, const double *fe, double *heat)
{
    double *U = (double *)malloc((size_t)n * sizeof(double) + 8);
    double *W = (double *)malloc((size_t)9 * n * sizeof(double) + 8);
    for (int step = 0; step < n_steps; ++step) {
        for (int i = 0; i < n; ++i) {
            double im = ORACLE_ACC / masses[types[i]];
            for (int k = 0; k < 3; ++k) {
                vel[(size_t)k * n + i] += 0.5 * dt * force[(size_t)k * n + i] * im;
                double x = pos[(size_t)k * n + i] + dt * vel[(size_t)k * n + i];
                pos[(size_t)k * n + i] = pbc[k] ? wrap1(x, box[k]) : x;
            }
        }
        double e, vt[9];
        if (oracle_compute(T, nR, nA, KR, KA, L, L4, L5, H, rcR, rcA, cR, cA, w0, b0, w1, b1, n, types, pos, box, pbc,
                           use_cells, NULL, 0, 0, &e, vt, U, force, W, NULL)) {
            free(U); free(W);
            return -1;
        }
        if (fe) oracle_hnemd_force(n, fe, W, force);
        double ke = 0.0;
        for (int i = 0; i < n; ++i) {
            double mi = masses[types[i]], im = ORACLE_ACC / mi;
            for (int k = 0; k < 3; ++k) {
                vel[(size_t)k * n + i] += 0.5 * dt * force[(size_t)k * n + i] * im;
                ke += 0.5 * mi * vel[(size_t)k * n + i] * vel[(size_t)k * n + i];
            }
        }
        if (noise) {
            double K = ke / ORACLE_ACC;  /* eV */
            double nf = 3.0 * n - 3.0, c = exp(-dt / tau), kbar = 0.5 * nf * 8.617333262e-5 * temperature;
            double r1 = noise[2 * step], chi = noise[2 * step + 1];
            double Kn = c * K + (1.0 - c) * kbar / nf * (r1 * r1 + chi) + 2.0 * r1 * sqrt(c * (1.0 - c) * K * kbar / nf);
            double alpha = (K > 0.0 && Kn > 0.0) ? sqrt(Kn / K) : (K > 0.0 ? 0.0 : 1.0);
            for (size_t k = 0; k < (size_t)3 * n; ++k) vel[k] *= alpha;
            ke *= alpha * alpha;
        }
        if (thermo) {
            thermo[2 * step] = e;
            thermo[2 * step + 1] = ke / ORACLE_ACC;
        }
        if (heat) oracle_heat_current(n, types, masses, vel, U, W, heat + (size_t)6 * step);
    }
    free(U); free(W);
    return 0;
}

/*
 * Coarse-grained mapping (Sec. II.B-C): bead position as the mass-weighted centre
 * of its atoms (Eq. 9), bead force and virial as sums over its atoms (Eq. 12,
 * Eq. 14).  Groups in CSR form (start[n_cg + 1], atoms[]).  On periodic axes each
 * atom is taken at its image nearest to the group's first atom; the centre is
 * wrapped into [0, L).  force / virial / outputs may be NULL.
 */
void oracle_cg_map(int n_cg, const int *start, const int *atoms, int n_aa, const double *mass, const double *pos,
                   const double *force, const double *virial, const double box[3], const int pbc[3],
                   double *bpos, double *bforce, double *bvirial)
{
    for (int I = 0; I < n_cg; ++I) {
        int a0 = atoms[start[I]];
        double msum = 0.0, c[3] = {0, 0, 0};
        for (int q = start[I]; q < start[I + 1]; ++q) {
            int i = atoms[q];
            msum += mass[i];
            for (int a = 0; a < 3; ++a) {
                double d = pos[(size_t)a * n_aa + i] - pos[(size_t)a * n_aa + a0];
                if (pbc[a]) d -= box[a] * round(d / box[a]);
                c[a] += mass[i] * (pos[(size_t)a * n_aa + a0] + d);
            }
        }
        if (bpos)
            for (int a = 0; a < 3; ++a) {
                double x = c[a] / msum;
                bpos[(size_t)a * n_cg + I] = pbc[a] ? wrap1(x, box[a]) : x;
            }
        if (bforce && force)
            for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int q = start[I]; q < start[I + 1]; ++q) s += force[(size_t)a * n_aa + atoms[q]];
                bforce[(size_t)a * n_cg + I] = s;
            }
        if (bvirial && virial)
            for (int k = 0; k < 9; ++k) {
                double s = 0.0;
                for (int q = start[I]; q < start[I + 1]; ++q) s += virial[(size_t)k * n_aa + atoms[q]];
                bvirial[(size_t)k * n_cg + I] = s;
            }
    }
}
