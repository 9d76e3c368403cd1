/*
 * FP64 oracle of the troubled-cell criterion and of the indicator network's input
 * features (TEST INFRASTRUCTURE ONLY; see dolinc_oracle.c).
 *
 * The paper has no troubled-cell criterion; this one is built only from quantities
 * the paper defines (reading stated in the design notes).  The paper cannot pin it;
 * its computation is pinned by closed forms in the tests (equal indicators of
 * quadratics on geometric strips, positivity of uniform states, the inputs of linear
 * fields on un-jittered triangles, the neighbour choice by brute force):
 * cell c is troubled if, at any of its faces,
 *   (i)  a reconstructed face state (either orientation, the scheme's fixed stencil)
 *        has density <= 0 or pressure <= 0, or
 *   (ii) for q in {rho, rho E}, with c as the upwind cell i and the far values
 *        phi_{-2..2} inverted by Eq diffDLC, the paper's three-cell ENO3 indicators
 *        (Sec 2.4) D_L = g^2 [phi_0 - (1+g) phi_-1 + g phi_-2],
 *        D_C = phi_1 - (1+g) phi_0 + g phi_-1, D_R = g^-2 [phi_2 - (1+g) phi_1 + g phi_0]
 *        satisfy |D_C| > kappa min(|D_L|, |D_R|) and |D_C| > eps (|phi_0| + |phi_1|).
 *
 * Features of cell c (6 per cell): for m = 1, 2 and each face f of c, the cell's own
 * DOLINC differential along the face, phi^(m)_c(d_f) = 2^m T^(m)_c : d_f^m (d_f from c
 * to its neighbour), of rho, of rho E and of the momentum vector (Euclidean norm of
 * its components); the maximum over faces is divided by rho_c, |E_c| and
 * sqrt(rho_c |E_c|) respectively and mapped by log(1 + x).  The 24 network inputs of
 * a cell are its own 6 followed by the 6 of three of its face neighbours (the cell
 * itself across a boundary face): the three largest in lexicographic order of their
 * 6 features, in decreasing order (so the input does not depend on face order).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int dim;
    long n_nodes, n_cells, n_faces;
    const double *nodes;
    const long *face_node_off;
    const long *face_nodes;
    const long *owner, *neigh;
    const double *shift;
} ind_mesh;

typedef struct {
    double *V, *xc, *S, *xf, *w, *d;
} ind_geom;

typedef struct {
    int nv, k, r, n_diff, flux;
    double gamma, adv[3];
    int eno;
    const unsigned char *troubled;
} ind_scheme;

/* from dolinc_oracle.c */
int or_phantoms(int N, double g, const double *phi0, const double *phi1, double *out);
int or_coeff(int k, int r, double g, double *c);

static int ipw(int b, int e) { int p = 1; while (e-- > 0) p *= b; return p; }

static long tofs(int D, int nv, long nc, int mm)
{
    long o = 0;
    for (int j = 0; j < mm; ++j) o += ipw(D, j);
    return o * nv * nc;
}

static double contract_full(int D, int mm, const double *Tm, const double *d)
{
    int A = ipw(D, mm);
    double s = 0.0;
    for (int a = 0; a < A; ++a) {
        double p = Tm[a];
        int t = a;
        for (int j = 0; j < mm; ++j) { p *= d[t % D]; t /= D; }
        s += p;
    }
    return ldexp(s, mm);
}

/* upwind geometry of face f seen from cell c (c is owner: side 0, neighbour: side 1) */
static void face_frame(const ind_mesh *m, const ind_geom *g, long f, int side, double *d, double *gr)
{
    long P = m->owner[f], Q = m->neigh[f];
    double sh[3] = {0, 0, 0}, xQ[3], a, b;
    if (m->shift) for (int k = 0; k < m->dim; ++k) sh[k] = m->shift[f * m->dim + k];
    for (int k = 0; k < 3; ++k) xQ[k] = g->xc[3*Q + k] + sh[k];
    double ra[3], rb[3];
    for (int k = 0; k < 3; ++k) { ra[k] = xQ[k] - g->xf[3*f + k]; rb[k] = g->xf[3*f + k] - g->xc[3*P + k]; }
    a = sqrt(ra[0]*ra[0] + ra[1]*ra[1] + ra[2]*ra[2]);
    b = sqrt(rb[0]*rb[0] + rb[1]*rb[1] + rb[2]*rb[2]);
    for (int k = 0; k < 3; ++k) d[k] = side == 0 ? xQ[k] - g->xc[3*P + k] : g->xc[3*P + k] - xQ[k];
    *gr = side == 0 ? a / b : b / a;
}

static double pressure(int D, double gam, const double *U)
{
    double ke = 0.0;
    for (int k = 0; k < D; ++k) ke += U[1 + k] * U[1 + k];
    return (gam - 1.0) * (U[D + 1] - 0.5 * ke / U[0]);
}

/* Criterion flags [n_cells] (Euler, nv = dim + 2, n_diff >= 2). */
int or_criterion(const ind_mesh *m, const ind_geom *g, const ind_scheme *s, const double *T, double kappa,
                 double eps, unsigned char *flags)
{
    const int D = m->dim, nv = s->nv, N = s->n_diff;
    const long nc = m->n_cells;
    double c[16], ph[16], p0[8], p1[8];
    if (N < 2 || nv != D + 2) return -1;
    memset(flags, 0, (size_t)nc);
    for (long f = 0; f < m->n_faces; ++f) {
        long P = m->owner[f], Q = m->neigh[f];
        if (Q < 0) continue;
        for (int side = 0; side < 2; ++side) {
            long i = side == 0 ? P : Q, j = side == 0 ? Q : P;
            double d[3], gr, U[8] = {0};
            face_frame(m, g, f, side, d, &gr);
            or_coeff(s->k, s->r, gr, c);
            int trouble = 0;
            for (int v = 0; v < nv; ++v) {
                for (int mm = 0; mm <= N; ++mm) {
                    const double *Tm = T + tofs(D, nv, nc, mm);
                    long A = ipw(D, mm);
                    p0[mm] = contract_full(D, mm, &Tm[((long)v * nc + i) * A], d);
                    p1[mm] = contract_full(D, mm, &Tm[((long)v * nc + j) * A], d);
                }
                or_phantoms(N, gr, p0, p1, ph);
                double val = 0.0;
                for (int q = 0; q < s->k; ++q) val += c[q] * ph[N + q - s->r];
                U[v] = val;
                if (v == 0 || v == nv - 1) {
                    const double *x = &ph[N - 2];          /* phi_{-2} .. phi_2 */
                    double DL = gr * gr * (x[2] - (1.0 + gr) * x[1] + gr * x[0]);
                    double DC = x[3] - (1.0 + gr) * x[2] + gr * x[1];
                    double DR = (x[4] - (1.0 + gr) * x[3] + gr * x[2]) / (gr * gr);
                    double mn = fabs(DL) < fabs(DR) ? fabs(DL) : fabs(DR);
                    if (fabs(DC) > kappa * mn && fabs(DC) > eps * (fabs(x[2]) + fabs(x[3]))) trouble = 1;
                }
            }
            if (!(U[0] > 0.0) || !(pressure(D, s->gamma, U) > 0.0)) { flags[P] = 1; flags[Q] = 1; }
            if (trouble) flags[i] = 1;
        }
    }
    return 0;
}

/* a > b in lexicographic order of the 6 features */
static int lex_greater(const double *a, const double *b)
{
    for (int q = 0; q < 6; ++q) {
        if (a[q] > b[q]) return 1;
        if (a[q] < b[q]) return 0;
    }
    return 0;
}

/* Own features [n_cells][6] and network inputs [n_cells][24] (Euler, n_diff >= 2). */
int or_indicator_features(const ind_mesh *m, const ind_geom *g, const ind_scheme *s, const double *T, double tiny,
                          double *own, double *x24)
{
    const int D = m->dim, nv = s->nv;
    const long nc = m->n_cells;
    long *off = calloc((size_t)nc + 1, sizeof(long));
    if (!off) return -1;
    for (long f = 0; f < m->n_faces; ++f) {
        off[m->owner[f] + 1]++;
        if (m->neigh[f] >= 0) off[m->neigh[f] + 1]++;
    }
    for (long c = 0; c < nc; ++c) off[c + 1] += off[c];
    long *nbr = malloc(sizeof(long) * (size_t)off[nc]);
    long *fill = malloc(sizeof(long) * (size_t)nc);
    if (!nbr || !fill) return -1;
    for (long c = 0; c < nc; ++c) fill[c] = off[c];
    for (long c = 0; c < nc * 6; ++c) own[c] = 0.0;
    for (long f = 0; f < m->n_faces; ++f) {
        long P = m->owner[f], Q = m->neigh[f];
        for (int side = 0; side < (Q >= 0 ? 2 : 1); ++side) {
            long c = side == 0 ? P : Q;
            nbr[fill[c]++] = Q < 0 ? P : (side == 0 ? Q : P);
            double d[3], gr;
            if (Q < 0) {
                for (int k = 0; k < 3; ++k) d[k] = 2.0 * (g->xf[3*f + k] - g->xc[3*P + k]);
            } else {
                face_frame(m, g, f, side, d, &gr);
            }
            for (int mm = 1; mm <= 2; ++mm) {
                const double *Tm = T + tofs(D, nv, nc, mm);
                long A = ipw(D, mm);
                double r = fabs(contract_full(D, mm, &Tm[(0L * nc + c) * A], d));
                double e = fabs(contract_full(D, mm, &Tm[((long)(nv - 1) * nc + c) * A], d));
                double mo = 0.0;
                for (int k = 0; k < D; ++k) {
                    double t = contract_full(D, mm, &Tm[((long)(1 + k) * nc + c) * A], d);
                    mo += t * t;
                }
                mo = sqrt(mo);
                double *o = &own[6 * c + 3 * (mm - 1)];
                if (r > o[0]) o[0] = r;
                if (e > o[1]) o[1] = e;
                if (mo > o[2]) o[2] = mo;
            }
        }
    }
    for (long c = 0; c < nc; ++c) {
        double rho = T[c], E = fabs(T[(long)(nv - 1) * nc + c]);
        double sc[3] = {rho + tiny, E + tiny, sqrt(fabs(rho) * E) + tiny};
        for (int mm = 0; mm < 2; ++mm)
            for (int q = 0; q < 3; ++q) own[6 * c + 3 * mm + q] = log1p(own[6 * c + 3 * mm + q] / sc[q]);
    }
    for (long c = 0; c < nc; ++c) {
        long top[3] = {c, c, c};
        int have = 0;
        for (long a = off[c]; a < off[c + 1]; ++a) {
            long o = nbr[a];
            /* insert o into the descending top-3 list */
            int pos = have < 3 ? have : 3;
            while (pos > 0 && lex_greater(&own[6 * o], &own[6 * top[pos - 1]])) {
                if (pos < 3) top[pos] = top[pos - 1];
                --pos;
            }
            if (pos < 3) top[pos] = o;
            if (have < 3) ++have;
        }
        for (int q = 0; q < 6; ++q) x24[24 * c + q] = own[6 * c + q];
        for (int a = 0; a < 3; ++a)
            for (int q = 0; q < 6; ++q) x24[24 * c + 6 + 6 * a + q] = own[6 * top[a] + q];
    }
    free(nbr);
    free(fill);
    free(off);
    return 0;
}
