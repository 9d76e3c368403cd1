/*
 * Plain FP64 CPU oracle of one DOLINC explicit Runge-Kutta stage on an
 * unstructured finite-volume mesh (arXiv 2404.08952).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this file's library.  It shares no code with the CUDA
 * library: it computes its own geometry, keeps FULL (unsymmetrised) Gauss tensors
 * of every differential order, obtains far-field values by the paper's recursion
 * in the paper's order, and builds reconstruction weights from the Lagrange
 * primitive formula itself.  Loops are face-centric scatters written for reading,
 * not for speed.
 *
 * Paper passages followed (section / equation of the paper):
 *   Sec 2.1            owner/neighbour face addressing
 *   Sec 2.2 Eqs 1-4    growth rate g, centre distance d, weight omega, g = omega/(1-omega)
 *   Sec 2.3            central-differencing (Gauss + linear interpolation) gradient,
 *                      Eq recursion, DOLINC differential definition, Eq diffDLC,
 *                      first/second-order inversion (Eqs lCoeffDLC1 .. rCoeffDLC2)
 *   Sec 2.4 Eq coeff   k-th order reconstruction weights c_rj on non-uniform cells
 *   Sec 2.4            ENO3-DOLINC smoothness indicators
 *   Sec 2.6            boundary handling (zero-gradient auxiliary cell)
 *   Sec 3              third-order TVD (SSP) Runge-Kutta; upwind, local Lax-Friedrichs
 *                      (Rusanov) and Roe fluxes
 *
 * Readings taken where the paper is silent (each is listed with its reason in the
 * design notes): Euclidean distances in Eq 3; cell averages (Eq 5 read with the
 * 1/dx factor); multi-dimensional differentials are the cell's m-fold Gauss tensor
 * contracted m times with the face's d; zero-gradient boundary faces take the
 * cell value as face value for every order; one flux point per face.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXD 3
#define OR_MAXN 4      /* highest differential order */
#define OR_MAXK 10     /* widest stencil: k <= 2N+2 */
#define OR_MAXV 5

typedef struct {
    int dim;
    long n_nodes, n_cells, n_faces;
    const double *nodes;            /* [n_nodes][dim] */
    const long *face_node_off;      /* [n_faces+1] */
    const long *face_nodes;
    const long *owner, *neigh;      /* neigh < 0: boundary face */
    const double *shift;            /* [n_faces][dim] neighbour translation, may be NULL */
} or_mesh;

typedef struct {
    double *V;    /* [n_cells]           cell volume (area in 2D) */
    double *xc;   /* [n_cells][3]        cell centroid */
    double *S;    /* [n_faces][3]        face area vector, out of the owner */
    double *xf;   /* [n_faces][3]        face centroid (owner side) */
    double *w;    /* [n_faces]           Eq 3 weight of the owner */
    double *d;    /* [n_faces][3]        Eq 2 centre distance, owner -> neighbour */
    /* skewness correction (NULL: the plain scheme), from or_skew_geometry */
    double *Minv; /* [n_cells][3][3]     inverse of the cell's skewness matrix M_c */
    double *sdelta; /* [n_faces][3]      face centroid minus the reconstruction point x* */
} or_geom;

typedef struct {
    int nv;           /* number of variables */
    int k, r;         /* stencil: k cells starting at i-r (Eq coeff) */
    int n_diff;       /* differential orders computed */
    int flux;         /* 0 linear advection upwind, 1 Burgers Roe, 2 Euler Rusanov */
    double gamma;     /* ratio of specific heats (Euler) */
    double adv[3];    /* advection velocity (flux 0) */
    int eno;          /* 0 fixed stencil, 1 ENO3 on every face, 2 ENO3 on faces touching a troubled cell,
                         3 first-order upwind (the cell's own average) on faces touching a troubled cell,
                         4 WENO5 on every face, 5 WENO5 on faces touching a troubled cell */
    const unsigned char *troubled;   /* [n_cells] for eno == 2, 3, 5 */
    const int *bkind;                /* [n_faces] boundary kind per face (NULL: every boundary face
                                        zero-gradient): 0/1 zero-gradient, 2 Dirichlet, 3 Neumann */
    const double *bval;              /* [nv][n_faces]: the face value (2) or the outward normal
                                        gradient (3) */
} or_scheme;

static int ipow(int b, int e) { int p = 1; while (e-- > 0) p *= b; return p; }

static void vsub(const double *a, const double *b, double *o) { for (int k = 0; k < 3; ++k) o[k] = a[k] - b[k]; }
static double vdot(const double *a, const double *b) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }
static double vnorm(const double *a) { return sqrt(vdot(a, a)); }
static void vcross(const double *a, const double *b, double *o)
{
    o[0] = a[1]*b[2] - a[2]*b[1];
    o[1] = a[2]*b[0] - a[0]*b[2];
    o[2] = a[0]*b[1] - a[1]*b[0];
}

static void node3(const or_mesh *m, long n, double *x)
{
    x[0] = x[1] = x[2] = 0.0;
    for (int k = 0; k < m->dim; ++k) x[k] = m->nodes[n * m->dim + k];
}

static void shift3(const or_mesh *m, long f, double *s)
{
    s[0] = s[1] = s[2] = 0.0;
    if (m->shift && m->neigh[f] >= 0)
        for (int k = 0; k < m->dim; ++k) s[k] = m->shift[f * m->dim + k];
}

/* Sub-triangles of a face, as seen from its owner: area vectors St and centroids ct.
 * 2D: the face is an edge a->b with area vector (b_y-a_y, -(b_x-a_x)).
 * 3D: a triangle is itself; a polygon is split into the triangles joining each
 * edge to the mean of its nodes.  Returns the number of pieces. */
static int face_pieces(const or_mesh *m, long f, double St[][3], double ct[][3])
{
    long o = m->face_node_off[f], n = m->face_node_off[f + 1] - o;
    if (m->dim == 2) {
        double a[3], b[3];
        node3(m, m->face_nodes[o], a);
        node3(m, m->face_nodes[o + 1], b);
        St[0][0] = b[1] - a[1]; St[0][1] = -(b[0] - a[0]); St[0][2] = 0.0;
        for (int k = 0; k < 3; ++k) ct[0][k] = 0.5 * (a[k] + b[k]);
        return 1;
    }
    if (n == 3) {
        double a[3], b[3], c[3], ab[3], ac[3];
        node3(m, m->face_nodes[o], a);
        node3(m, m->face_nodes[o + 1], b);
        node3(m, m->face_nodes[o + 2], c);
        vsub(b, a, ab); vsub(c, a, ac);
        vcross(ab, ac, St[0]);
        for (int k = 0; k < 3; ++k) { St[0][k] *= 0.5; ct[0][k] = (a[k] + b[k] + c[k]) / 3.0; }
        return 1;
    }
    double mc[3] = {0, 0, 0}, p[3];
    for (long e = 0; e < n; ++e) { node3(m, m->face_nodes[o + e], p); for (int k = 0; k < 3; ++k) mc[k] += p[k] / (double)n; }
    for (long e = 0; e < n; ++e) {
        double a[3], b[3], am[3], bm[3];
        node3(m, m->face_nodes[o + e], a);
        node3(m, m->face_nodes[o + (e + 1) % n], b);
        vsub(a, mc, am); vsub(b, mc, bm);
        vcross(am, bm, St[e]);
        for (int k = 0; k < 3; ++k) { St[e][k] *= 0.5; ct[e][k] = (mc[k] + a[k] + b[k]) / 3.0; }
    }
    return (int)n;
}

/* Geometry (Sec 2.2).  Cells are the polyhedra (polygons) bounded by the face
 * pieces above; a periodic face's neighbour side is the owner side moved by -shift. */
int or_geometry(const or_mesh *m, or_geom *g)
{
    const int D = m->dim;
    double (*St)[3] = malloc(sizeof(double[64][3]));
    double (*ct)[3] = malloc(sizeof(double[64][3]));
    double *cnt = calloc((size_t)m->n_cells, sizeof(double));
    double *apex = calloc((size_t)m->n_cells * 3, sizeof(double));
    if (!St || !ct || !cnt || !apex) return -1;
    memset(g->V, 0, sizeof(double) * (size_t)m->n_cells);
    memset(g->xc, 0, sizeof(double) * 3 * (size_t)m->n_cells);
    for (long f = 0; f < m->n_faces; ++f) {
        int np = face_pieces(m, f, St, ct);
        double S[3] = {0, 0, 0}, xf[3] = {0, 0, 0}, area = 0.0;
        for (int t = 0; t < np; ++t) {
            double a = vnorm(St[t]);
            for (int k = 0; k < 3; ++k) { S[k] += St[t][k]; xf[k] += a * ct[t][k]; }
            area += a;
        }
        for (int k = 0; k < 3; ++k) { g->S[3*f + k] = S[k]; g->xf[3*f + k] = xf[k] / area; }
    }
    /* apex of each cell: mean of its face centroids in its own frame */
    for (long f = 0; f < m->n_faces; ++f) {
        long P = m->owner[f], N = m->neigh[f];
        double s[3];
        shift3(m, f, s);
        for (int k = 0; k < 3; ++k) apex[3*P + k] += g->xf[3*f + k];
        cnt[P] += 1.0;
        if (N >= 0) {
            for (int k = 0; k < 3; ++k) apex[3*N + k] += g->xf[3*f + k] - s[k];
            cnt[N] += 1.0;
        }
    }
    for (long c = 0; c < m->n_cells; ++c) for (int k = 0; k < 3; ++k) apex[3*c + k] /= cnt[c];
    /* volumes and centroids from pyramids (apex, face piece) */
    for (long f = 0; f < m->n_faces; ++f) {
        int np = face_pieces(m, f, St, ct);
        long P = m->owner[f], N = m->neigh[f];
        double s[3];
        shift3(m, f, s);
        for (int side = 0; side < (N >= 0 ? 2 : 1); ++side) {
            long c = side == 0 ? P : N;
            double sg = side == 0 ? 1.0 : -1.0;
            for (int t = 0; t < np; ++t) {
                double cc[3], rel[3], St_out[3];
                for (int k = 0; k < 3; ++k) { cc[k] = ct[t][k] - (side ? s[k] : 0.0); St_out[k] = sg * St[t][k]; }
                vsub(cc, &apex[3*c], rel);
                double vol = vdot(St_out, rel) / (double)D;
                g->V[c] += vol;
                for (int k = 0; k < 3; ++k) g->xc[3*c + k] += vol * (apex[3*c + k] + D * cc[k]) / (double)(D + 1);
            }
        }
    }
    for (long c = 0; c < m->n_cells; ++c) for (int k = 0; k < 3; ++k) g->xc[3*c + k] /= g->V[c];
    /* Eq 3 weight and Eq 2 distance, Euclidean, with the periodic translation */
    for (long f = 0; f < m->n_faces; ++f) {
        long P = m->owner[f], N = m->neigh[f];
        const double *xf = &g->xf[3*f];
        if (N < 0) {
            g->w[f] = 1.0;
            for (int k = 0; k < 3; ++k) g->d[3*f + k] = 2.0 * (xf[k] - g->xc[3*P + k]);
            continue;
        }
        double s[3], xN[3], a[3], b[3];
        shift3(m, f, s);
        for (int k = 0; k < 3; ++k) xN[k] = g->xc[3*N + k] + s[k];
        vsub(xN, xf, a);
        vsub(&g->xc[3*P], xf, b);
        g->w[f] = vnorm(a) / (vnorm(b) + vnorm(a));
        for (int k = 0; k < 3; ++k) g->d[3*f + k] = xN[k] - g->xc[3*P + k];
    }
    free(St); free(ct); free(cnt); free(apex);
    return 0;
}

/* Skewness correction (the paper names the low accuracy of its inversion on
 * tetrahedral and hybrid grids as future work, Sec 4; this correction is this
 * library's).  The linear interpolation of Eq 3 gives the face the value of a linear
 * field at x*_f = x_P + (1 - w) d, the point of the centroid line that divides it like
 * the face, and the DOLINC reconstruction along d is likewise a value at x*_f; on a
 * skewed mesh x*_f is not the face centroid x_f.  For a linear field the Gauss sum of
 * such face values is M_c grad(phi) with
 *   M_c = (1/V_c) sum_f S_{c,f} (x) (x*_f - x_c)      (M_c = I when every x*_f = x_f),
 * so the corrected pass applies M_c^-1 to the new (gradient) index of every order, and
 * the face value gets the shift (x_f - x*_f) . T^(1) of its upwind cell.  Both are
 * exact for linear fields on meshes with planar faces.  Boundary faces count as
 * unskewed (x*_f = x_f).  Fills g->Minv and g->sdelta (allocated by the caller);
 * returns -1 if some M_c is singular. */
int or_skew_geometry(const or_mesh *m, or_geom *g)
{
    const int D = m->dim;
    const long nc = m->n_cells;
    double *M = calloc((size_t)nc * 9, sizeof(double));
    if (!M) return -1;
    for (long f = 0; f < m->n_faces; ++f) {
        long P = m->owner[f], N = m->neigh[f];
        const double *S = &g->S[3*f], *xf = &g->xf[3*f];
        double xs[3], sh[3];
        shift3(m, f, sh);
        for (int k = 0; k < 3; ++k)
            xs[k] = N >= 0 ? g->xc[3*P + k] + (1.0 - g->w[f]) * g->d[3*f + k] : xf[k];
        for (int k = 0; k < 3; ++k) g->sdelta[3*f + k] = xf[k] - xs[k];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                M[9*P + 3*i + j] += S[i] * (xs[j] - g->xc[3*P + j]) / g->V[P];
                if (N >= 0) M[9*N + 3*i + j] -= S[i] * (xs[j] - sh[j] - g->xc[3*N + j]) / g->V[N];
            }
    }
    for (long c = 0; c < nc; ++c) {
        double *a = &M[9*c], *b = &g->Minv[9*c];
        if (D == 2) { a[2] = a[5] = a[6] = a[7] = 0.0; a[8] = 1.0; }
        /* inverse by cofactors */
        double det = a[0] * (a[4]*a[8] - a[5]*a[7]) - a[1] * (a[3]*a[8] - a[5]*a[6]) + a[2] * (a[3]*a[7] - a[4]*a[6]);
        if (!(fabs(det) > 1e-12)) { free(M); return -1; }
        b[0] = (a[4]*a[8] - a[5]*a[7]) / det; b[1] = (a[2]*a[7] - a[1]*a[8]) / det; b[2] = (a[1]*a[5] - a[2]*a[4]) / det;
        b[3] = (a[5]*a[6] - a[3]*a[8]) / det; b[4] = (a[0]*a[8] - a[2]*a[6]) / det; b[5] = (a[2]*a[3] - a[0]*a[5]) / det;
        b[6] = (a[3]*a[7] - a[4]*a[6]) / det; b[7] = (a[1]*a[6] - a[0]*a[7]) / det; b[8] = (a[0]*a[4] - a[1]*a[3]) / det;
    }
    free(M);
    return 0;
}

/* offset of differential order mm in the concatenated full-tensor buffer */
static long toff(int D, int nv, long nc, int mm)
{
    long o = 0;
    for (int j = 0; j < mm; ++j) o += (long)ipow(D, j);
    return o * nv * nc;
}

/* Value of variable v on boundary face f of cell P (Sec 2.6): the prescribed value
 * on a Dirichlet face; T_C + q delta on a Neumann face, q the outward normal gradient
 * and delta the distance from the cell centroid to the face along the outward unit
 * normal; the cell value on a zero-gradient face. */
static double boundary_value(const or_geom *g, const int *bkind, const double *bval, long n_faces, long f, long P,
                             int v, double tP)
{
    const int kind = bkind ? bkind[f] : 1;
    if (kind == 2) return bval[(long)v * n_faces + f];
    if (kind == 3) {
        const double *S = &g->S[3*f];
        double r[3];
        vsub(&g->xf[3*f], &g->xc[3*P], r);
        return tP + bval[(long)v * n_faces + f] * vdot(r, S) / vnorm(S);
    }
    return tP;
}

/* DOLINC differentials, Sec 2.3: T^(0) is the cell average; T^(m) is the
 * central-differencing (Gauss, linearly interpolated) gradient of T^(m-1):
 *   T^(m)_c = (1/V_c) sum_f S_{c,f} (x) [ w T^(m-1)_c + (1-w) T^(m-1)_nb ].
 * The new gradient index is the leading one.  Boundary faces (Sec 2.6): the first
 * gradient takes the boundary face value (boundary_value); higher orders take the
 * cell's own differential (the auxiliary cell beyond the face carries the boundary
 * cell's differentials).  Buffer: order m at toff(m), laid out [v][c][D^m]. */
int or_differentials_bc(const or_mesh *m, const or_geom *g, int nv, int N, const double *u, const int *bkind,
                        const double *bval, double *T);

int or_differentials(const or_mesh *m, const or_geom *g, int nv, int N, const double *u, double *T)
{
    return or_differentials_bc(m, g, nv, N, u, NULL, NULL, T);
}

/* One Gauss pass: order mm (>= 1) from order mm-1, full tensors [v][c][D^(mm-1)] ->
 * [v][c][D^mm]; boundary faces as in or_differentials_bc. */
int or_gauss_pass(const or_mesh *m, const or_geom *g, int nv, int mm, const double *Ti, double *To, const int *bkind,
                  const double *bval)
{
    const int D = m->dim;
    const long nc = m->n_cells;
    if (mm < 1 || mm > OR_MAXN) return -1;
    const int Ain = ipow(D, mm - 1), Aout = ipow(D, mm);
    memset(To, 0, sizeof(double) * (size_t)nv * (size_t)nc * (size_t)Aout);
    for (long f = 0; f < m->n_faces; ++f) {
        long P = m->owner[f], Q = m->neigh[f];
        const double *S = &g->S[3*f];
        double w = g->w[f];
        for (int v = 0; v < nv; ++v)
            for (int a = 0; a < Ain; ++a) {
                double tP = Ti[((long)v * nc + P) * Ain + a];
                double tf = Q >= 0 ? w * tP + (1.0 - w) * Ti[((long)v * nc + Q) * Ain + a]
                                   : (mm == 1 ? boundary_value(g, bkind, bval, m->n_faces, f, P, v, tP) : tP);
                for (int k = 0; k < D; ++k) {
                    To[((long)v * nc + P) * Aout + k * Ain + a] += S[k] * tf / g->V[P];
                    if (Q >= 0) To[((long)v * nc + Q) * Aout + k * Ain + a] -= S[k] * tf / g->V[Q];
                }
            }
    }
    if (g->Minv) {              /* skewness correction: M_c^-1 on the new index */
        for (int v = 0; v < nv; ++v)
            for (long c = 0; c < nc; ++c)
                for (int a = 0; a < Ain; ++a) {
                    double t[3] = {0.0, 0.0, 0.0}, o[3];
                    for (int k = 0; k < D; ++k) t[k] = To[((long)v * nc + c) * Aout + k * Ain + a];
                    for (int k = 0; k < D; ++k) {
                        o[k] = 0.0;
                        for (int j = 0; j < D; ++j) o[k] += g->Minv[9*c + 3*k + j] * t[j];
                    }
                    for (int k = 0; k < D; ++k) To[((long)v * nc + c) * Aout + k * Ain + a] = o[k];
                }
    }
    return 0;
}

int or_differentials_bc(const or_mesh *m, const or_geom *g, int nv, int N, const double *u, const int *bkind,
                        const double *bval, double *T)
{
    const int D = m->dim;
    const long nc = m->n_cells;
    memcpy(T, u, sizeof(double) * (size_t)nv * (size_t)nc);
    for (int mm = 1; mm <= N; ++mm)
        or_gauss_pass(m, g, nv, mm, T + toff(D, nv, nc, mm - 1), T + toff(D, nv, nc, mm), bkind, bval);
    return 0;
}

/* DOLINC differential of a cell along d (Sec 2.3):
 * varphi^(m) = 2^m T_{j1..jm} d_j1 ... d_jm, summed over every index tuple. */
static double contract(int D, int mm, const double *Tm, const double *d)
{
    int A = ipow(D, mm);
    double s = 0.0;
    for (int a = 0; a < A; ++a) {
        double p = Tm[a];
        int t = a;
        for (int j = 0; j < mm; ++j) { p *= d[t % D]; t /= D; }
        s += p;
    }
    return ldexp(s, mm);
}

/* Eq coeff: k-th order reconstruction weights at x_{i+1/2} from the cell averages
 * of cells i-r .. i-r+k-1, on cells that grow by the constant factor g (Eq 1).
 * Cell i has unit width, cell i+n width g^n; x_{i+1/2} = 0. */
static double face_pos(double g, int n)   /* right face of cell i+n */
{
    double x = 0.0;
    if (n >= 0) { for (int j = 1; j <= n; ++j) x += pow(g, j); }
    else        { for (int j = n + 1; j <= 0; ++j) x -= pow(g, j); }
    return x;
}

int or_coeff(int k, int r, double g, double *c)
{
    double x[OR_MAXK + 1];
    if (k < 1 || k > OR_MAXK || r < 0 || r >= k) return -1;
    for (int q = 0; q <= k; ++q) x[q] = face_pos(g, -r + q - 1);   /* x_{i-r+q-1/2} */
    const double xf = 0.0;                                          /* x_{i+1/2} */
    for (int j = 0; j < k; ++j) {
        double s = 0.0;
        for (int mq = j + 1; mq <= k; ++mq) {
            double num = 0.0, den = 1.0;
            for (int l = 0; l <= k; ++l) {
                if (l == mq) continue;
                double p = 1.0;
                for (int q = 0; q <= k; ++q) if (q != mq && q != l) p *= (xf - x[q]);
                num += p;
                den *= (x[mq] - x[l]);
            }
            s += num / den;
        }
        c[j] = s * (x[j + 1] - x[j]);                               /* times dx_{i-r+j} */
    }
    return 0;
}

/* Far-field values by Eq diffDLC,
 *   phi_{n+1}^(m) - g phi_{n-1}^(m) = g^n phi_n^(m+1) + (1-g) phi_n^(m),
 * applied outward from the two face cells (n = 0, 1) in the paper's order:
 * forward for n >= 2 (Eq recursion form), backward for n <= -1.
 * phi0[m], phi1[m] (m = 0..N) are the upwind and downwind cells' differentials.
 * out[n + N] = phi_n^(0) for n = -N .. N+1 (2N+2 values). */
int or_phantoms(int N, double g, const double *phi0, const double *phi1, double *out)
{
    double tab[2 * OR_MAXN + 2][OR_MAXN + 1];
    if (N < 0 || N > OR_MAXN) return -1;
    const int o = N;              /* tab[n + o][m] */
    for (int mm = 0; mm <= N; ++mm) { tab[o][mm] = phi0[mm]; tab[o + 1][mm] = phi1[mm]; }
    for (int n = 2; n <= N + 1; ++n)               /* centre n-1 */
        for (int mm = 0; mm <= N - (n - 1); ++mm)
            tab[n + o][mm] = g * tab[n - 2 + o][mm] + pow(g, n - 1) * tab[n - 1 + o][mm + 1]
                           + (1.0 - g) * tab[n - 1 + o][mm];
    for (int n = -1; n >= -N; --n)                 /* centre n+1 */
        for (int mm = 0; mm <= N + n; ++mm)
            tab[n + o][mm] = (tab[n + 2 + o][mm] - pow(g, n + 1) * tab[n + 1 + o][mm + 1]
                              - (1.0 - g) * tab[n + 1 + o][mm]) / g;
    for (int n = -N; n <= N + 1; ++n) out[n + N] = tab[n + o][0];
    return 0;
}

/* ENO3-DOLINC (Sec 2.4): classical two-level stencil growth with the paper's
 * non-uniform divided-difference indicators.  Ties: level 2 keeps the upwind
 * side {i-1, i}; level 3 keeps the centred stencil {i-1, i, i+1}.
 * ph[n+2] = phi_n for n = -2..2.  Returns the chosen r (0, 1 or 2). */
static int eno3_choose(double g, const double *ph)
{
    const double p_2 = ph[0], p_1 = ph[1], p0 = ph[2], p1 = ph[3], p2 = ph[4];
    double d2l = g * (p0 - p_1), d2r = p1 - p0;
    double dL = g * g * (p0 - (1.0 + g) * p_1 + g * p_2);
    double dC = p1 - (1.0 + g) * p0 + g * p_1;
    double dR = (p2 - (1.0 + g) * p1 + g * p0) / (g * g);
    if (fabs(d2l) <= fabs(d2r)) return fabs(dL) < fabs(dC) ? 2 : 1;
    return fabs(dR) < fabs(dC) ? 0 : 1;
}

/* WENO5-DOLINC (Sec 2.4 names it: the fixed stencils plus stencil weights).  The
 * three 3-cell candidates r = 0, 1, 2 (Eq coeff weights on the geometric cells) are
 * combined with the nonlinear weights of Jiang and Shu,
 *   w_r = a_r / sum a,  a_r = d_r / (1e-6 + beta_r)^2,
 * where the linear weights d_r make the combination the 5-cell stencil (5, 2) (they
 * follow from its two end coefficients: only r = 2 reaches cell i-2 and only r = 0
 * cell i+2), and beta_r is the Jiang-Shu smoothness measure of the candidate's
 * quadratic p_r on the upwind cell, in units of that cell's width:
 *   beta_r = int_cell (p_r')^2 + (p_r'')^2 dx,
 * p_r the derivative of the cubic interpolating the primitive at the candidate's four
 * faces.  On uniform cells this is the classical WENO5.  ph[n+2] = phi_n, n = -2..2.
 * or_weno5_parts returns the candidate values q[r], the linear weights d[r] and the
 * smoothness beta[r] (r = 0, 1, 2); weno5_value combines them. */
int or_weno5_parts(double g, const double *ph, double *q, double *d, double *beta)
{
    double c5[5], c3[3];
    if (!(g > 0.0)) return -1;
    or_coeff(5, 2, g, c5);
    for (int r = 0; r < 3; ++r) {
        or_coeff(3, r, g, c3);
        q[r] = 0.0;
        for (int j = 0; j < 3; ++j) q[r] += c3[j] * ph[2 + j - r];
        if (r == 2) d[2] = c5[0] / c3[0];
        if (r == 0) d[0] = c5[4] / c3[2];
        /* primitive at the candidate's faces X_0..X_3 (cells i-r .. i-r+2) */
        double X[4], Pf[4] = {0.0, 0.0, 0.0, 0.0};
        for (int t = 0; t < 4; ++t) X[t] = face_pos(g, -r + t - 1);
        for (int t = 1; t < 4; ++t) Pf[t] = Pf[t - 1] + ph[2 - r + t - 1] * (X[t] - X[t - 1]);
        /* cubic P = a0 + a1 x + a2 x^2 + a3 x^3 through (X_t, Pf_t): Vandermonde solve */
        double A[4][5];
        for (int t = 0; t < 4; ++t) {
            double xp = 1.0;
            for (int e = 0; e < 4; ++e) { A[t][e] = xp; xp *= X[t]; }
            A[t][4] = Pf[t];
        }
        for (int col = 0; col < 4; ++col) {                /* Gaussian elimination, partial pivoting */
            int piv = col;
            for (int t = col + 1; t < 4; ++t) if (fabs(A[t][col]) > fabs(A[piv][col])) piv = t;
            for (int e = 0; e < 5; ++e) { double tmp = A[col][e]; A[col][e] = A[piv][e]; A[piv][e] = tmp; }
            for (int t = 0; t < 4; ++t) {
                if (t == col) continue;
                double f = A[t][col] / A[col][col];
                for (int e = col; e < 5; ++e) A[t][e] -= f * A[col][e];
            }
        }
        const double a2 = A[2][4] / A[2][2], a3 = A[3][4] / A[3][3];
        /* p' = 2 a2 + 6 a3 x, p'' = 6 a3 over the upwind cell [-1, 0] */
        const double b = 2.0 * a2, cc = 6.0 * a3;
        beta[r] = (b * b - b * cc + cc * cc / 3.0) + cc * cc;   /* int_{-1}^{0} (b + cc x)^2 dx + cc^2 */
    }
    d[1] = 1.0 - d[0] - d[2];
    return 0;
}

/* The WENO5-DOLINC face value: the candidates q_r weighted by the normalised
 * a_r = d_r / (1e-6 + beta_r)^2 (parts from or_weno5_parts). */
static double weno5_value(double g, const double *ph)
{
    double q[3], d[3], beta[3];
    or_weno5_parts(g, ph, q, d, beta);
    double a[3], sa = 0.0;
    for (int r = 0; r < 3; ++r) { a[r] = d[r] / ((1e-6 + beta[r]) * (1e-6 + beta[r])); sa += a[r]; }
    return (a[0] * q[0] + a[1] * q[1] + a[2] * q[2]) / sa;
}

/* Face value of one variable for one orientation (upwind cell i, downwind i+1);
 * use_eno: 1 ENO3-DOLINC, 2 WENO5-DOLINC. */
static double reconstruct(const or_scheme *s, int N, double g, const double *phi0, const double *phi1, int use_eno,
                          int *r_used)
{
    double ph[2 * OR_MAXN + 2], c[OR_MAXK];
    or_phantoms(N, g, phi0, phi1, ph);
    int k = s->k, r = s->r;
    if (use_eno == 2) {
        if (r_used) *r_used = -2;
        return weno5_value(g, &ph[N - 2]);
    }
    if (use_eno) { k = 3; r = eno3_choose(g, &ph[N - 2]); }
    if (r_used) *r_used = r;
    or_coeff(k, r, g, c);
    double v = 0.0;
    for (int j = 0; j < k; ++j) v += c[j] * ph[N + j - r];
    return v;
}

/* Both orientations of every variable at face f: L = owner upwind, R = neighbour upwind. */
static void face_states(const or_mesh *m, const or_geom *g, const or_scheme *s, const double *T,
                        long f, double *UL, double *UR, int *rL, int *rR)
{
    const int D = m->dim, nv = s->nv, N = s->n_diff;
    const long nc = m->n_cells;
    long P = m->owner[f], Q = m->neigh[f];
    if (Q < 0) {
        for (int v = 0; v < nv; ++v) {
            UL[v] = UR[v] = boundary_value(g, s->bkind, s->bval, m->n_faces, f, P, v, T[(long)v * nc + P]);
            if (rL) rL[v] = rR[v] = -1;
        }
        return;
    }
    double sh[3], xQ[3], dL[3], dR[3], a[3], b[3];
    const double *xf = &g->xf[3*f];
    shift3(m, f, sh);
    for (int k = 0; k < 3; ++k) xQ[k] = g->xc[3*Q + k] + sh[k];
    vsub(xQ, &g->xc[3*P], dL);                  /* owner upwind: d = x_{i+1} - x_i */
    vsub(&g->xc[3*P], xQ, dR);                  /* neighbour upwind */
    vsub(xQ, xf, a); vsub(xf, &g->xc[3*P], b);
    double gL = vnorm(a) / vnorm(b);            /* Eq 4 from the owner */
    double gR = vnorm(b) / vnorm(a);            /* Eq 4 from the neighbour */
    const int touched = s->troubled && (s->troubled[P] || s->troubled[Q]);
    if (s->eno == 3 && touched) {
        /* first-order fallback: each orientation takes its upwind cell's average */
        for (int v = 0; v < nv; ++v) {
            UL[v] = T[(long)v * nc + P];
            UR[v] = T[(long)v * nc + Q];
            if (rL) rL[v] = rR[v] = 0;
        }
        return;
    }
    int eno = (s->eno == 1 || (s->eno == 2 && touched)) ? 1 : (s->eno == 4 || (s->eno == 5 && touched)) ? 2 : 0;
    for (int v = 0; v < nv; ++v) {
        double pP[OR_MAXN + 1], pQ[OR_MAXN + 1], qP[OR_MAXN + 1], qQ[OR_MAXN + 1];
        for (int mm = 0; mm <= N; ++mm) {
            const double *Tm = T + toff(D, nv, nc, mm);
            long A = ipow(D, mm);
            pP[mm] = contract(D, mm, &Tm[((long)v * nc + P) * A], dL);
            pQ[mm] = contract(D, mm, &Tm[((long)v * nc + Q) * A], dL);
            qQ[mm] = contract(D, mm, &Tm[((long)v * nc + Q) * A], dR);
            qP[mm] = contract(D, mm, &Tm[((long)v * nc + P) * A], dR);
        }
        UL[v] = reconstruct(s, N, gL, pP, pQ, eno, rL ? &rL[v] : NULL);
        UR[v] = reconstruct(s, N, gR, qQ, qP, eno, rR ? &rR[v] : NULL);
        if (g->sdelta) {        /* skewness correction: from x*_f to the face centroid */
            const double *T1 = T + toff(D, nv, nc, 1), *dl = &g->sdelta[3*f];
            for (int k = 0; k < D; ++k) {
                UL[v] += dl[k] * T1[((long)v * nc + P) * D + k];
                UR[v] += dl[k] * T1[((long)v * nc + Q) * D + k];
            }
        }
    }
}

static void euler_phys(int D, double gam, const double *U, const double *S, double *F, double *un, double *c)
{
    double rho = U[0], ke = 0.0, vn = 0.0, Sn = 0.0;
    for (int k = 0; k < D; ++k) { double vk = U[1 + k] / rho; ke += vk * U[1 + k]; vn += vk * S[k]; Sn += S[k] * S[k]; }
    double E = U[D + 1];
    double p = (gam - 1.0) * (E - 0.5 * ke);
    F[0] = rho * vn;
    for (int k = 0; k < D; ++k) F[1 + k] = U[1 + k] * vn + p * S[k];
    F[D + 1] = (E + p) * vn;
    *un = vn / sqrt(Sn);
    *c = sqrt(gam * p / rho);
}

/* Numerical flux through S (owner -> neighbour) from the two reconstructed states. */
static void num_flux(int D, const or_scheme *s, const double *UL, const double *UR, const double *S, double *F)
{
    if (s->flux == 0) {
        double an = 0.0;
        for (int k = 0; k < D; ++k) an += s->adv[k] * S[k];
        F[0] = an * (an >= 0.0 ? UL[0] : UR[0]);
    } else if (s->flux == 1) {
        double sg = 0.0;
        for (int k = 0; k < D; ++k) sg += S[k];
        double lam = 0.5 * (UL[0] + UR[0]) * sg;      /* Roe speed of f(u) = u^2/2 (1,..,1) */
        double uu = lam >= 0.0 ? UL[0] : UR[0];
        F[0] = 0.5 * uu * uu * sg;
    } else {
        double FL[OR_MAXV], FR[OR_MAXV], unL, unR, cL, cR;
        euler_phys(D, s->gamma, UL, S, FL, &unL, &cL);
        euler_phys(D, s->gamma, UR, S, FR, &unR, &cR);
        double a = fmax(fabs(unL) + cL, fabs(unR) + cR);
        double Sn = sqrt(vdot(S, S));
        for (int v = 0; v < D + 2; ++v) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * a * Sn * (UR[v] - UL[v]);
    }
}

/* num_flux for a caller: dimension D, scheme s (flux, gamma, adv), states UL, UR of
 * s->nv variables and the face area vector S (owner -> neighbour); F gets s->nv values. */
int or_num_flux(int D, const or_scheme *s, const double *UL, const double *UR, const double *S, double *F)
{
    if (D < 1 || D > OR_MAXD || s->nv < 1 || s->nv > OR_MAXV) return -1;
    double S3[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < D; ++k) S3[k] = S[k];
    num_flux(D, s, UL, UR, S3, F);
    return 0;
}

/* Reconstructed face states of every face: [v][f] for L (owner upwind) and R. */
int or_face_values(const or_mesh *m, const or_geom *g, const or_scheme *s, const double *T,
                   double *phiL, double *phiR, int *rL, int *rR)
{
    const int nv = s->nv;
    for (long f = 0; f < m->n_faces; ++f) {
        double UL[OR_MAXV], UR[OR_MAXV];
        int a[OR_MAXV], b[OR_MAXV];
        face_states(m, g, s, T, f, UL, UR, a, b);
        for (int v = 0; v < nv; ++v) {
            phiL[(long)v * m->n_faces + f] = UL[v];
            phiR[(long)v * m->n_faces + f] = UR[v];
            if (rL) { rL[(long)v * m->n_faces + f] = a[v]; rR[(long)v * m->n_faces + f] = b[v]; }
        }
    }
    return 0;
}

/* Residual R_c = -(1/V_c) sum_f (+-) F_f from differentials T (Sec 3): every face's
 * flux first, then the sums over faces in face order.  The face fluxes are
 * independent of one another; a build with OpenMP (-fopenmp) computes them on all
 * threads, with the same results (the sums stay sequential). */
int or_residual_T(const or_mesh *m, const or_geom *g, const or_scheme *s, const double *T, double *R)
{
    const int D = m->dim, nv = s->nv;
    const long nc = m->n_cells, nf = m->n_faces;
    double *Ff = malloc(sizeof(double) * (size_t)nv * (size_t)(nf > 0 ? nf : 1));
    if (!Ff) return -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4096)
#endif
    for (long f = 0; f < nf; ++f) {
        double UL[OR_MAXV], UR[OR_MAXV];
        face_states(m, g, s, T, f, UL, UR, NULL, NULL);
        num_flux(D, s, UL, UR, &g->S[3*f], &Ff[f * nv]);
    }
    memset(R, 0, sizeof(double) * (size_t)nv * (size_t)nc);
    for (long f = 0; f < nf; ++f) {
        long P = m->owner[f], Q = m->neigh[f];
        const double *F = &Ff[f * nv];
        for (int v = 0; v < nv; ++v) {
            R[(long)v * nc + P] -= F[v] / g->V[P];
            if (Q >= 0) R[(long)v * nc + Q] += F[v] / g->V[Q];
        }
    }
    free(Ff);
    return 0;
}

static long tsize(int D, int nv, long nc, int N) { return toff(D, nv, nc, N + 1); }

int or_residual(const or_mesh *m, const or_geom *g, const or_scheme *s, const double *u, double *R)
{
    double *T = malloc(sizeof(double) * (size_t)tsize(m->dim, s->nv, m->n_cells, s->n_diff));
    if (!T) return -1;
    or_differentials_bc(m, g, s->nv, s->n_diff, u, s->bkind, s->bval, T);
    int rc = or_residual_T(m, g, s, T, R);
    free(T);
    return rc;
}

/* Threads the build computes face fluxes on: 1 without OpenMP. */
int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* One step of the third-order TVD (SSP) Runge-Kutta scheme (Sec 3):
 *   u1 = u + dt R(u);  u2 = 3/4 u + 1/4 (u1 + dt R(u1));  u' = 1/3 u + 2/3 (u2 + dt R(u2)). */
int or_rk3_step(const or_mesh *m, const or_geom *g, const or_scheme *s, double dt, double *u)
{
    const long n = (long)s->nv * m->n_cells;
    double *u1 = malloc(sizeof(double) * (size_t)n), *R = malloc(sizeof(double) * (size_t)n);
    if (!u1 || !R) return -1;
    int rc = or_residual(m, g, s, u, R);
    for (long i = 0; i < n; ++i) u1[i] = u[i] + dt * R[i];
    rc |= or_residual(m, g, s, u1, R);
    for (long i = 0; i < n; ++i) u1[i] = 0.75 * u[i] + 0.25 * (u1[i] + dt * R[i]);
    rc |= or_residual(m, g, s, u1, R);
    for (long i = 0; i < n; ++i) u[i] = u[i] / 3.0 + 2.0 / 3.0 * (u1[i] + dt * R[i]);
    free(u1); free(R);
    return rc ? -1 : 0;
}

/* One stage as the fused GPU stage computes it: given the step's start u0 and the
 * stage input us, return  a*u0 + b*(us + dt R(us))  with (a, b) = (0,1), (3/4,1/4), (1/3,2/3). */
int or_rk3_stage(const or_mesh *m, const or_geom *g, const or_scheme *s, double dt, int stage,
                 const double *u0, const double *us, double *out)
{
    static const double A[3] = {0.0, 0.75, 1.0 / 3.0}, B[3] = {1.0, 0.25, 2.0 / 3.0};
    const long n = (long)s->nv * m->n_cells;
    double *R = malloc(sizeof(double) * (size_t)n);
    if (!R || stage < 0 || stage > 2) { free(R); return -1; }
    int rc = or_residual(m, g, s, us, R);
    for (long i = 0; i < n; ++i) out[i] = A[stage] * u0[i] + B[stage] * (us[i] + dt * R[i]);
    free(R);
    return rc;
}

/* Conditioning of each face value: the weights W0[m], W1[m] (m = 0..N) of the DOLINC
 * representation  phi_f = sum_m W0[m] phi_0^(m) + W1[m] phi_1^(m)  (Sec 2.4, Eq USR3
 * generalised), obtained by running the oracle's own recursion (or_phantoms) on unit
 * data and weighting with or_coeff.  Used by the tests to scale parity tolerances by
 * sum |W| (large growth rates amplify rounding like g^N).  Output per face:
 * WL[f][2(N+1)] for the owner-upwind orientation, WR for the neighbour-upwind one,
 * W0 first then W1.  Boundary faces get W0[0] = 1. */
int or_face_weights(const or_mesh *m, const or_geom *g, const or_scheme *s, double *WL, double *WR)
{
    const int N = s->n_diff, nw = 2 * (N + 1);
    double c[OR_MAXK], e0[OR_MAXN + 1], e1[OR_MAXN + 1], ph[2 * OR_MAXN + 2];
    for (long f = 0; f < m->n_faces; ++f) {
        long P = m->owner[f], Q = m->neigh[f];
        for (int o = 0; o < 2; ++o) {
            double *W = (o == 0 ? WL : WR) + f * nw;
            for (int i = 0; i < nw; ++i) W[i] = 0.0;
            if (Q < 0) { W[0] = 1.0; continue; }
            double sh[3], xQ[3], a[3], b[3];
            const double *xf = &g->xf[3*f];
            shift3(m, f, sh);
            for (int k = 0; k < 3; ++k) xQ[k] = g->xc[3*Q + k] + sh[k];
            vsub(xQ, xf, a); vsub(xf, &g->xc[3*P], b);
            double gg = o == 0 ? vnorm(a) / vnorm(b) : vnorm(b) / vnorm(a);
            or_coeff(s->k, s->r, gg, c);
            for (int side = 0; side < 2; ++side)
                for (int mm = 0; mm <= N; ++mm) {
                    for (int q = 0; q <= N; ++q) { e0[q] = 0.0; e1[q] = 0.0; }
                    if (side == 0) e0[mm] = 1.0; else e1[mm] = 1.0;
                    or_phantoms(N, gg, e0, e1, ph);
                    double w = 0.0;
                    for (int j = 0; j < s->k; ++j) w += c[j] * ph[N + j - s->r];
                    W[side * (N + 1) + mm] = w;
                }
        }
    }
    return 0;
}
