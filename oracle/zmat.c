/*
 * oracle/zmat.c -- plain FP64 reference for the RWG-level PMCHWT operators.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this code.  The product
 * library never links it and shares no code with it.
 *
 * What is computed (paper Sec. II-B, Eqs. (K), (T) and the RHS definitions,
 * Galerkin testing with the RWG functions themselves):
 *
 *   K_i[m][n] = int_{t_m} int_{f_n} t_m(r) . ( grad G_i(r,r') x f_n(r') ) dr' dr
 *   T_i[m][n] = -j k_i int int G_i(r,r') [ t_m . f_n - (div t_m)(div' f_n)/k_i^2 ] dr' dr
 *   v^E[m]    =  int t_m . E_inc,        v^H[m] = - int t_m . H_inc
 *
 * with G_i = exp(-j k_i R)/(4 pi R), grad G_i = g_i(R)(r - r'),
 * g_i(R) = -(1 + j k_i R) exp(-j k_i R)/(4 pi R^3).  The testing identity
 * (n x t).(n x X) = t.X for tangential t is used.  The minus sign on T is the
 * reading under which the paper's block matrix [[K, -eta T], [T/eta, K]] and
 * right-hand side [n x E_inc; -n x H_inc] describe the e^{+j omega t}
 * problem with J = n x H, M = E x n (Sec. II-A, Eqs. (1)-(2), (10)-(12)).
 *
 * Quadrature (the paper does not fix it): the 7-point degree-5 rule on every
 * triangle, test and trial.  A triangle pair is "near" when it shares a vertex
 * or its centroid distance is below alpha * max(longest edge).  Near pairs use
 * singularity extraction: 1/R (for T) and 1/R^3 + k^2/(2R) (for K) are
 * integrated analytically over the trial triangle at each test point, the
 * bounded remainders with the 7-point rule.  The K block of a triangle with
 * itself is zero (flat triangle: the triple product vanishes).  Near-pair
 * local blocks are symmetrised: L(t,t')[a][b] = (L~(t,t')[a][b] + L~(t',t)[b][a])/2.
 *
 * Mesh convention: local edge a of triangle t joins vertices (a+1)%3 and
 * (a+2)%3 and has free vertex a.  sign = +1 when t is the edge's plus triangle.
 * RWG on t: f = sign * l / (2 A_t) * (r - p_a).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define PI 3.14159265358979323846

/* ---------------------------------------------------------------- vectors */
static inline void sub3(const double *a, const double *b, double *c) { c[0] = a[0]-b[0]; c[1] = a[1]-b[1]; c[2] = a[2]-b[2]; }
static inline double dot3(const double *a, const double *b) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }
static inline void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1]*b[2] - a[2]*b[1]; c[1] = a[2]*b[0] - a[0]*b[2]; c[2] = a[0]*b[1] - a[1]*b[0];
}
static inline double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* ------------------------------------------------- 7-point degree-5 rule
 * Radon's rule (Strang & Fix table): centroid weight 9/40; two orbits of
 * three points (a,b,b) with b = (6 -/+ sqrt15)/21, weights (155 -/+ sqrt15)/1200.
 * Weights sum to one; multiply by the triangle area. */
void orc_quad7_bary(double bary[7][3], double w[7]) {
    const double s15 = sqrt(15.0);
    const double b1 = (6.0 - s15) / 21.0, a1 = 1.0 - 2.0 * b1;
    const double b2 = (6.0 + s15) / 21.0, a2 = 1.0 - 2.0 * b2;
    const double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
    double B[7][3] = {{1.0/3, 1.0/3, 1.0/3},
                      {a1, b1, b1}, {b1, a1, b1}, {b1, b1, a1},
                      {a2, b2, b2}, {b2, a2, b2}, {b2, b2, a2}};
    double W[7] = {9.0/40.0, w1, w1, w1, w2, w2, w2};
    memcpy(bary, B, sizeof(B));
    memcpy(w, W, sizeof(W));
}

typedef struct {
    double v[3][3];     /* vertices */
    double n[3];        /* unit normal */
    double area;
    double c[3];        /* centroid */
    double h;           /* longest edge */
    double q[7][3];     /* quadrature points */
    double w[7];        /* weights * area */
} tri_t;

static void make_tri(const double *verts, const int *tri, tri_t *T) {
    double bary[7][3], w[7];
    orc_quad7_bary(bary, w);
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) T->v[a][d] = verts[3 * tri[a] + d];
    double e1[3], e2[3], e3[3], nn[3];
    sub3(T->v[1], T->v[0], e1);
    sub3(T->v[2], T->v[0], e2);
    sub3(T->v[2], T->v[1], e3);
    cross3(e1, e2, nn);
    double nl = norm3(nn);
    T->area = 0.5 * nl;
    for (int d = 0; d < 3; ++d) T->n[d] = nn[d] / nl;
    for (int d = 0; d < 3; ++d) T->c[d] = (T->v[0][d] + T->v[1][d] + T->v[2][d]) / 3.0;
    double h = norm3(e1);
    if (norm3(e2) > h) h = norm3(e2);
    if (norm3(e3) > h) h = norm3(e3);
    T->h = h;
    for (int p = 0; p < 7; ++p) {
        for (int d = 0; d < 3; ++d)
            T->q[p][d] = bary[p][0] * T->v[0][d] + bary[p][1] * T->v[1][d] + bary[p][2] * T->v[2][d];
        T->w[p] = w[p] * T->area;
    }
}

/* ------------------------------------------ analytic potential integrals
 * For a flat triangle S with vertices v0,v1,v2 (counter-clockwise about its
 * normal n) and an observation point r, returns
 *   I1    = int_S 1/R dS'
 *   Iv    = int_S (r' - r)/R dS'
 *   I3    = int_S (r - r')/R^3 dS'   (Cauchy principal value when r lies in S)
 * using the edge-sum closed forms of Wilton et al. (IEEE TAP 1984) and
 * Graglia (IEEE TAP 1993): with rho the projection of r on the plane,
 * d = n.(r - v0), and per edge the unit direction l, outward in-plane normal
 * u = l x n, signed distance t0 = (A - rho).u, l+- = (B/A - rho).l,
 * R0^2 = t0^2 + d^2, R+- = |r - B/A|, F = ln((R+ + l+)/(R- + l-)):
 *   I1 = sum t0 F - |d| sum beta,  beta = atan(t0 l+/(R0^2+|d|R+)) - atan(t0 l-/(R0^2+|d|R-))
 *   int (rho' - rho)/R = 1/2 sum u [R0^2 F + l+ R+ - l- R-]
 *   int (rho - rho')/R^3 = sum u F,   n.int (r - r')/R^3 = sign(d) sum beta
 */
static double log_rpl(double l, double R, double R02) {
    /* ln(R + l), stable for l < 0 via (R+l)(R-l) = R0^2 */
    if (l >= 0.0) return log(R + l);
    return log(R02 / (R - l));
}

void orc_potentials(const double *v0, const double *v1, const double *v2, const double *r,
                    double *I1, double *Iv, double *I3) {
    const double *V[3] = {v0, v1, v2};
    double e1[3], e2[3], n[3];
    sub3(v1, v0, e1);
    sub3(v2, v0, e2);
    cross3(e1, e2, n);
    double nl = norm3(n);
    for (int d = 0; d < 3; ++d) n[d] /= nl;
    double rv0[3];
    sub3(r, v0, rv0);
    double dd = dot3(n, rv0);
    double ad = fabs(dd);
    double rho[3] = {r[0] - dd * n[0], r[1] - dd * n[1], r[2] - dd * n[2]};
    double scale = sqrt(nl);            /* ~ edge length */
    double tiny = 1e-28 * scale * scale;
    double sumF_t0 = 0.0, sumbeta = 0.0;
    double vecrho[3] = {0, 0, 0}, vecF[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i) {
        const double *A = V[i], *B = V[(i + 1) % 3];
        double lv[3];
        sub3(B, A, lv);
        double ll = norm3(lv);
        for (int d = 0; d < 3; ++d) lv[d] /= ll;
        double u[3];
        cross3(lv, n, u);
        double Ar[3], Br[3];
        sub3(A, rho, Ar);
        sub3(B, rho, Br);
        double t0 = dot3(Ar, u);
        double lp = dot3(Br, lv), lm = dot3(Ar, lv);
        double R02 = t0 * t0 + dd * dd;
        double rA[3], rB[3];
        sub3(r, A, rA);
        sub3(r, B, rB);
        double Rp = norm3(rB), Rm = norm3(rA);
        double F = 0.0;
        if (R02 > tiny) F = log_rpl(lp, Rp, R02) - log_rpl(lm, Rm, R02);
        double beta = 0.0;
        if (ad > 0.0)
            beta = atan(t0 * lp / (R02 + ad * Rp)) - atan(t0 * lm / (R02 + ad * Rm));
        sumF_t0 += t0 * F;
        sumbeta += beta;
        double coef = 0.5 * (R02 * F + lp * Rp - lm * Rm);
        for (int d = 0; d < 3; ++d) {
            vecrho[d] += coef * u[d];
            vecF[d] += F * u[d];
        }
    }
    double i1 = sumF_t0 - ad * sumbeta;
    *I1 = i1;
    double sg = (dd > 0.0) ? 1.0 : ((dd < 0.0) ? -1.0 : 0.0);
    for (int d = 0; d < 3; ++d) {
        Iv[d] = vecrho[d] - dd * n[d] * i1;
        I3[d] = vecF[d] + n[d] * sg * sumbeta;
    }
}

/* ---------------------------------------------- smooth kernel remainders */
/* G_s(R) = (exp(-jkR) - 1)/(4 pi R); value at R = 0 is -jk/(4 pi). */
static cplx green_smooth(cplx k, double R) {
    cplx x = -I * k * R;
    if (cabs(x) < 0.5) {
        /* (e^x - 1)/R = k' sum_{m>=1} x^{m-1}/m!  with x = -jkR */
        cplx term = 1.0, s = 0.0;
        for (int m = 1; m < 30; ++m) {
            term = (m == 1) ? 1.0 : term * x / m;   /* x^{m-1}/m! built incrementally */
            s += term;
        }
        /* s = sum_{m>=1} x^{m-1}/m!  (recurrence above: term_m = x^{m-1}/m!) */
        return (-I * k) * s / (4.0 * PI);
    }
    return (cexp(x) - 1.0) / (4.0 * PI * R);
}

/* g_s(R) = g(R) + 1/(4 pi R^3) + k^2/(8 pi R); value at R = 0 is j k^3/(12 pi). */
static cplx gradgreen_smooth(cplx k, double R) {
    cplx x = I * k * R;
    if (cabs(x) < 0.5) {
        /* (1+x)e^{-x} - 1 + x^2/2 = sum_{m>=3} (-1)^m (1-m)/m! x^m, divided by R^3 */
        cplx s = 0.0;
        cplx kx = I * k;                 /* x/R */
        cplx pw = kx * kx * kx;          /* (x/R)^3 */
        double fact = 6.0;
        for (int m = 3; m < 34; ++m) {
            if (m > 3) { pw *= x; fact *= m; }
            /* pw = (jk)^3 x^{m-3} = x^m / R^3 */
            double cm = ((m % 2) ? -1.0 : 1.0) * (1.0 - m) / fact;
            s += cm * pw;
        }
        return -s / (4.0 * PI);
    }
    cplx g = -(1.0 + I * k * R) * cexp(-I * k * R) / (4.0 * PI * R * R * R);
    return g + 1.0 / (4.0 * PI * R * R * R) + k * k / (8.0 * PI * R);
}

/* ------------------------------------------------ local 3x3 blocks */
typedef struct {
    const double *verts;
    const int *tris;
    const int *tri_sign;     /* nt*3 */
    const double *edge_len;  /* ne   */
    const int *tri_edge;     /* nt*3 */
    int nt;
    tri_t *T;
    double alpha;
} mesh_t;

static int shares_vertex(const int *a, const int *b) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (a[i] == b[j]) return 1;
    return 0;
}

int orc_is_near(const mesh_t *M, int t, int s) {
    if (shares_vertex(M->tris + 3 * t, M->tris + 3 * s)) return 1;
    double dc[3];
    sub3(M->T[t].c, M->T[s].c, dc);
    double h = M->T[t].h > M->T[s].h ? M->T[t].h : M->T[s].h;
    return norm3(dc) < M->alpha * h;
}

static void local_coef(const mesh_t *M, int t, double c[3], const double *p[3]) {
    for (int a = 0; a < 3; ++a) {
        int e = M->tri_edge[3 * t + a];
        c[a] = M->tri_sign[3 * t + a] * M->edge_len[e] / (2.0 * M->T[t].area);
        p[a] = M->T[t].v[a];
    }
}

/* Plain 7x7 double sum, direct vector form of the integrands. */
static void block_far(const mesh_t *M, int t, int s, cplx k, cplx Kl[3][3], cplx Tl[3][3]) {
    const tri_t *A = &M->T[t], *B = &M->T[s];
    double ca[3], cb[3];
    const double *pa[3], *pb[3];
    local_coef(M, t, ca, pa);
    local_coef(M, s, cb, pb);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Kl[a][b] = Tl[a][b] = 0.0;
    for (int p = 0; p < 7; ++p) {
        for (int q = 0; q < 7; ++q) {
            double d[3];
            sub3(A->q[p], B->q[q], d);
            double R = norm3(d);
            cplx e = cexp(-I * k * R);
            cplx G = e / (4.0 * PI * R);
            cplx g = -(1.0 + I * k * R) * e / (4.0 * PI * R * R * R);
            double ww = A->w[p] * B->w[q];
            for (int a = 0; a < 3; ++a) {
                double ta[3];
                sub3(A->q[p], pa[a], ta);            /* t / c_a */
                for (int b = 0; b < 3; ++b) {
                    double fb[3], cr[3];
                    sub3(B->q[q], pb[b], fb);        /* f / c_b */
                    cross3(d, fb, cr);               /* (r - r') x f */
                    double cc = ca[a] * cb[b];
                    Kl[a][b] += ww * cc * g * dot3(ta, cr);
                    Tl[a][b] += ww * cc * (-I * k) * G * (dot3(ta, fb) - 4.0 / (k * k));
                }
            }
        }
    }
}

/* Singularity-extracted block: outer 7 points on t, inner analytic + 7 points on s. */
static void block_near_raw(const mesh_t *M, int t, int s, cplx k, cplx Kl[3][3], cplx Tl[3][3]) {
    const tri_t *A = &M->T[t], *B = &M->T[s];
    double ca[3], cb[3];
    const double *pa[3], *pb[3];
    local_coef(M, t, ca, pa);
    local_coef(M, s, cb, pb);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Kl[a][b] = Tl[a][b] = 0.0;
    for (int p = 0; p < 7; ++p) {
        const double *r = A->q[p];
        double I1, Iv[3], I3[3];
        orc_potentials(B->v[0], B->v[1], B->v[2], r, &I1, Iv, I3);
        /* S0 = int G, S1[b] = int G (r' - p_b), W = int g (r - r') */
        cplx S0 = I1 / (4.0 * PI);
        cplx Sr[3];           /* int G (r' - r) */
        cplx W[3];
        for (int d = 0; d < 3; ++d) {
            Sr[d] = Iv[d] / (4.0 * PI);
            W[d] = -I3[d] / (4.0 * PI) + k * k / (8.0 * PI) * Iv[d];
        }
        for (int q = 0; q < 7; ++q) {
            double d[3];
            sub3(r, B->q[q], d);
            double R = norm3(d);
            cplx gs = green_smooth(k, R);
            cplx hs = gradgreen_smooth(k, R);
            S0 += B->w[q] * gs;
            for (int x = 0; x < 3; ++x) {
                Sr[x] += B->w[q] * gs * (-d[x]);
                W[x] += B->w[q] * hs * d[x];
            }
        }
        for (int a = 0; a < 3; ++a) {
            double ta[3];
            sub3(r, pa[a], ta);
            for (int b = 0; b < 3; ++b) {
                double rb[3];
                sub3(r, pb[b], rb);                 /* r - p_b */
                /* int G (r' - p_b) = Sr + (r - p_b) S0 */
                cplx tdotS = 0.0;
                for (int x = 0; x < 3; ++x) tdotS += ta[x] * (Sr[x] + rb[x] * S0);
                double cc = ca[a] * cb[b];
                Tl[a][b] += A->w[p] * cc * (-I * k) * (tdotS - 4.0 / (k * k) * S0);
                if (t != s) {
                    /* (r - p_a) . (W x (r - p_b)) */
                    cplx cr[3];
                    cr[0] = W[1] * rb[2] - W[2] * rb[1];
                    cr[1] = W[2] * rb[0] - W[0] * rb[2];
                    cr[2] = W[0] * rb[1] - W[1] * rb[0];
                    Kl[a][b] += A->w[p] * cc * (ta[0] * cr[0] + ta[1] * cr[1] + ta[2] * cr[2]);
                }
            }
        }
    }
}

static void block(const mesh_t *M, int t, int s, cplx k, cplx Kl[3][3], cplx Tl[3][3]) {
    if (!orc_is_near(M, t, s)) {
        block_far(M, t, s, k, Kl, Tl);
        return;
    }
    cplx K1[3][3], T1[3][3], K2[3][3], T2[3][3];
    block_near_raw(M, t, s, k, K1, T1);
    block_near_raw(M, s, t, k, K2, T2);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            Kl[a][b] = 0.5 * (K1[a][b] + K2[b][a]);
            Tl[a][b] = 0.5 * (T1[a][b] + T2[b][a]);
        }
}

static void mesh_init(mesh_t *M, int nv, const double *verts, int nt, const int *tris,
                      const int *tri_edge, const int *tri_sign, const double *edge_len, double alpha) {
    (void)nv;
    M->verts = verts; M->tris = tris; M->tri_edge = tri_edge; M->tri_sign = tri_sign;
    M->edge_len = edge_len; M->nt = nt; M->alpha = alpha;
    M->T = (tri_t *)malloc(sizeof(tri_t) * (size_t)nt);
    for (int t = 0; t < nt; ++t) make_tri(verts, tris + 3 * t, &M->T[t]);
}

/* Local blocks of one triangle pair for one medium (row-major 3x3, interleaved re/im). */
void orc_local_block(int nv, const double *verts, int nt, const int *tris, const int *tri_edge,
                     const int *tri_sign, const double *edge_len, double alpha,
                     double k_re, double k_im, int t, int s, double *Kout, double *Tout, int *near) {
    mesh_t M;
    mesh_init(&M, nv, verts, nt, tris, tri_edge, tri_sign, edge_len, alpha);
    cplx k = k_re + I * k_im, Kl[3][3], Tl[3][3];
    block(&M, t, s, k, Kl, Tl);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            Kout[2 * (3 * a + b)] = creal(Kl[a][b]); Kout[2 * (3 * a + b) + 1] = cimag(Kl[a][b]);
            Tout[2 * (3 * a + b)] = creal(Tl[a][b]); Tout[2 * (3 * a + b) + 1] = cimag(Tl[a][b]);
        }
    *near = orc_is_near(&M, t, s);
    free(M.T);
}

/*
 * Dense RWG blocks K[rows][cols], T[rows][cols] for one medium.
 * Each entry is the sum over the 2 x 2 triangle pairs of the two supports:
 *   Z[i][j] = sum_{s,s'} L(t_i^s, t_j^s')[a_i^s][a_j^s'].
 * edge_tri/edge_loc: (ne, 2) plus/minus triangle and local index.
 * Output arrays are row-major (nrows, ncols) complex128.
 */
void orc_assemble(int nv, const double *verts, int nt, const int *tris, const int *tri_edge,
                  const int *tri_sign, const double *edge_len, const int *edge_tri, const int *edge_loc,
                  double alpha, double k_re, double k_im,
                  int nrows, const int *rows, int ncols, const int *cols,
                  cplx *Kout, cplx *Tout) {
    mesh_t M;
    mesh_init(&M, nv, verts, nt, tris, tri_edge, tri_sign, edge_len, alpha);
    cplx k = k_re + I * k_im;
    /* trial triangles touched by the column set */
    char *need = (char *)calloc((size_t)nt, 1);
    for (int c = 0; c < ncols; ++c) {
        need[edge_tri[2 * cols[c]]] = 1;
        need[edge_tri[2 * cols[c] + 1]] = 1;
    }
#pragma omp parallel
    {
        cplx *rowK = (cplx *)malloc(sizeof(cplx) * 3 * (size_t)nt);
        cplx *rowT = (cplx *)malloc(sizeof(cplx) * 3 * (size_t)nt);
#pragma omp for schedule(dynamic, 1)
        for (int ri = 0; ri < nrows; ++ri) {
            int i = rows[ri];
            for (int c = 0; c < ncols; ++c) { Kout[(size_t)ri * ncols + c] = 0.0; Tout[(size_t)ri * ncols + c] = 0.0; }
            for (int sgn = 0; sgn < 2; ++sgn) {
                int t = edge_tri[2 * i + sgn], a = edge_loc[2 * i + sgn];
                for (int s = 0; s < nt; ++s) {
                    if (!need[s]) continue;
                    cplx Kl[3][3], Tl[3][3];
                    block(&M, t, s, k, Kl, Tl);
                    for (int b = 0; b < 3; ++b) { rowK[3 * s + b] = Kl[a][b]; rowT[3 * s + b] = Tl[a][b]; }
                }
                for (int c = 0; c < ncols; ++c) {
                    int j = cols[c];
                    for (int sp = 0; sp < 2; ++sp) {
                        int s = edge_tri[2 * j + sp], b = edge_loc[2 * j + sp];
                        Kout[(size_t)ri * ncols + c] += rowK[3 * s + b];
                        Tout[(size_t)ri * ncols + c] += rowT[3 * s + b];
                    }
                }
            }
        }
        free(rowK);
        free(rowT);
    }
    free(need);
    free(M.T);
}

/* ------------------------------------------------------- plane waves */
static void sph_basis(double th, double ph, double rh[3], double thh[3], double phh[3]) {
    rh[0] = sin(th) * cos(ph); rh[1] = sin(th) * sin(ph); rh[2] = cos(th);
    thh[0] = cos(th) * cos(ph); thh[1] = cos(th) * sin(ph); thh[2] = -sin(th);
    phh[0] = -sin(ph); phh[1] = cos(ph); phh[2] = 0.0;
}

/*
 * RHS of the paper's Eq. (v): vE[e][w] = int f_e . E_inc, vH[e][w] = -int f_e . H_inc,
 * for unit-amplitude plane waves arriving from r_hat(theta, phi):
 *   k_hat = -r_hat, E_inc = p exp(-j k1 k_hat . r), H_inc = k_hat x E_inc / eta1,
 *   p = cos(psi) theta_hat + sin(psi) phi_hat.
 * Output (ne, nw) complex128.
 */
void orc_rhs(int nv, const double *verts, int nt, const int *tris, const int *tri_edge,
             const int *tri_sign, const double *edge_len, int ne, double k1, double eta1,
             int nw, const double *waves, cplx *vE, cplx *vH) {
    mesh_t M;
    mesh_init(&M, nv, verts, nt, tris, tri_edge, tri_sign, edge_len, 1.0);
    memset(vE, 0, sizeof(cplx) * (size_t)ne * nw);
    memset(vH, 0, sizeof(cplx) * (size_t)ne * nw);
    for (int w = 0; w < nw; ++w) {
        double rh[3], thh[3], phh[3];
        sph_basis(waves[3 * w], waves[3 * w + 1], rh, thh, phh);
        double kh[3] = {-rh[0], -rh[1], -rh[2]};
        double p[3], hp[3];
        for (int d = 0; d < 3; ++d) p[d] = cos(waves[3 * w + 2]) * thh[d] + sin(waves[3 * w + 2]) * phh[d];
        cross3(kh, p, hp);
        for (int t = 0; t < nt; ++t) {
            double ca[3];
            const double *pa[3];
            local_coef(&M, t, ca, pa);
            for (int q = 0; q < 7; ++q) {
                const double *r = M.T[t].q[q];
                cplx ph = cexp(-I * k1 * dot3(kh, r));
                for (int a = 0; a < 3; ++a) {
                    double f[3];
                    sub3(r, pa[a], f);
                    int e = M.tri_edge[3 * t + a];
                    vE[(size_t)e * nw + w] += M.T[t].w[q] * ca[a] * dot3(f, p) * ph;
                    vH[(size_t)e * nw + w] -= M.T[t].w[q] * ca[a] * dot3(f, hp) / eta1 * ph;
                }
            }
        }
    }
    free(M.T);
}

/*
 * Far-field pattern F(r_hat) with E_scat ~ F exp(-j k1 r)/r, radiated into the
 * exterior medium by J = sum aJ_e f_e and M = sum aM_e f_e:
 *   F = (j k1 / 4 pi) [ -eta1 (N - r_hat (r_hat . N)) + r_hat x L ],
 *   N = int J exp(j k1 r_hat . r'), L = int M exp(j k1 r_hat . r').
 * aM, aJ: (ne, nrhs); dirs (ndir, 2); F_th, F_ph out: (nrhs, ndir).
 */
void orc_farfield(int nv, const double *verts, int nt, const int *tris, const int *tri_edge,
                  const int *tri_sign, const double *edge_len, int ne, double k1, double eta1,
                  int nrhs, const cplx *aM, const cplx *aJ, int ndir, const double *dirs,
                  cplx *Fth, cplx *Fph) {
    (void)ne;
    mesh_t M;
    mesh_init(&M, nv, verts, nt, tris, tri_edge, tri_sign, edge_len, 1.0);
#pragma omp parallel for schedule(dynamic, 1)
    for (int dI = 0; dI < ndir; ++dI) {
        double rh[3], thh[3], phh[3];
        sph_basis(dirs[2 * dI], dirs[2 * dI + 1], rh, thh, phh);
        for (int w = 0; w < nrhs; ++w) {
            cplx N[3] = {0, 0, 0}, L[3] = {0, 0, 0};
            for (int t = 0; t < nt; ++t) {
                double ca[3];
                const double *pa[3];
                local_coef(&M, t, ca, pa);
                for (int q = 0; q < 7; ++q) {
                    const double *r = M.T[t].q[q];
                    cplx ph = cexp(I * k1 * dot3(rh, r)) * M.T[t].w[q];
                    for (int a = 0; a < 3; ++a) {
                        int e = M.tri_edge[3 * t + a];
                        double f[3];
                        sub3(r, pa[a], f);
                        cplx cJ = aJ[(size_t)e * nrhs + w] * ca[a] * ph;
                        cplx cM = aM[(size_t)e * nrhs + w] * ca[a] * ph;
                        for (int x = 0; x < 3; ++x) { N[x] += cJ * f[x]; L[x] += cM * f[x]; }
                    }
                }
            }
            /* theta / phi components */
            cplx Nth = N[0] * thh[0] + N[1] * thh[1] + N[2] * thh[2];
            cplx Nph = N[0] * phh[0] + N[1] * phh[1] + N[2] * phh[2];
            cplx Lth = L[0] * thh[0] + L[1] * thh[1] + L[2] * thh[2];
            cplx Lph = L[0] * phh[0] + L[1] * phh[1] + L[2] * phh[2];
            /* r x L = L_th phi_hat - L_ph theta_hat */
            cplx pre = I * k1 / (4.0 * PI);
            Fth[(size_t)w * ndir + dI] = pre * (-eta1 * Nth - Lph);
            Fph[(size_t)w * ndir + dI] = pre * (-eta1 * Nph + Lth);
        }
    }
    free(M.T);
}
