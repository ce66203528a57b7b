/*
 * FP64 CPU oracle: dense P1-Galerkin boundary operators of the linearised
 * Poisson-Boltzmann interface problem.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library; the product path never
 * does. It shares no code with the CUDA library.
 *
 * What it computes (paper, "Boundary integral formulations", layer potentials
 * and Green's functions; "Numerical discretization": P1 Galerkin, DOF = vertices):
 *   G_int(r) = 1/(4 pi r)                (Laplace, interior)
 *   G_ext(r) = exp(-kappa r)/(4 pi r)    (Yukawa, exterior)
 *   V_ij = int int phi_i(x) G(x,y) phi_j(y)                     single layer
 *   K_ij = int int phi_i(x) dG/dn_y(x,y) phi_j(y)               double layer
 *   D_ij = int int G(x,y) [curl phi_i(x).curl phi_j(y)
 *                          + kappa^2 n_x.n_y phi_i(x) phi_j(y)] hypersingular
 *                                                               (integrated by parts)
 *   T = K^T (adjoint double layer), M_ij = int phi_i phi_j (mass).
 * with dG/dn_y = (x-y).n_y (1 + kappa r) exp(-kappa r) / (4 pi r^3).
 *
 * Quadrature (the discrete definition shared with the GPU path by
 * specification, not by code):
 *   - triangle pairs sharing no vertex: the same symmetric triangle rule on
 *     both triangles (points/weights passed in by the caller); with a distance
 *     band (band_eta > 0), pairs whose centroids are closer than band_eta
 *     times the sum of their radii (largest centroid-vertex distance) take a
 *     second, finer rule instead, so that the coarse rule only meets pairs
 *     that are far apart relative to their size;
 *   - coincident, edge-adjacent and vertex-adjacent pairs: regularising maps
 *     of [0,1]^4 in the manner of Sauter and Schwab (6, 6 and 2 regions) with
 *     an n-point Gauss-Legendre rule per dimension (nodes/weights passed in),
 *     n chosen per class: ng[0] coincident, ng[1] edge, ng[2] vertex, the
 *     three rules' nodes (and weights) one after another in gx (gw).
 *
 * Reference triangle for the singular maps: T^ = {(s,t): 0 <= t <= s <= 1},
 * vertices (0,0), (1,0), (1,1); a triangle with reordered vertices (Q0,Q1,Q2)
 * is x(s,t) = Q0 + s (Q1-Q0) + t (Q2-Q1), barycentrics (1-s, s-t, t), and
 * |dx/d(s,t)| = 2|tau|.
 *
 * Assembly is a plain loop over all triangle pairs. It is parallelised over
 * test triangles of one colour at a time (no two triangles of a colour share
 * a vertex), so every matrix entry receives its terms in one fixed order and
 * the result does not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NOPS 6 /* V_L, K_L, D_L, V_Y, K_Y, D_Y */

typedef struct {
    double p[3][3];  /* vertex coordinates */
    double n[3];     /* unit outward normal (right-hand rule on the listed order) */
    double area;
    double e[3][3];  /* edge opposite local vertex a, counter-clockwise */
} tri_geom;

static const double PI = 3.14159265358979323846;

static void sub3(const double* a, const double* b, double* c) {
    c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2];
}
static double dot3(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static void make_geom(const double* verts, const int32_t* tri, tri_geom* g) {
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) g->p[a][k] = verts[3 * (int64_t)tri[a] + k];
    double u[3], v[3], c[3];
    sub3(g->p[1], g->p[0], u);
    sub3(g->p[2], g->p[0], v);
    cross3(u, v, c);
    double len = sqrt(dot3(c, c));
    g->area = 0.5 * len;
    for (int k = 0; k < 3; ++k) g->n[k] = c[k] / len;
    sub3(g->p[2], g->p[1], g->e[0]);
    sub3(g->p[0], g->p[2], g->e[1]);
    sub3(g->p[1], g->p[0], g->e[2]);
}

/* Both Green's functions and their y-normal derivatives at one point pair. */
typedef struct { double gl, gy, kl, ky; } kern_vals;

static kern_vals kernels(const double* x, const double* y, const double* ny, double kappa) {
    double d[3];
    sub3(x, y, d);
    double r = sqrt(dot3(d, d));
    double dn = dot3(d, ny);
    double inv4pir = 1.0 / (4.0 * PI * r);
    double ek = exp(-kappa * r);
    kern_vals kv;
    kv.gl = inv4pir;
    kv.gy = ek * inv4pir;
    kv.kl = dn * inv4pir / (r * r);
    kv.ky = ek * (1.0 + kappa * r) * dn * inv4pir / (r * r);
    return kv;
}

/* Add the weighted integrand of one point pair into the six 3x3 local blocks.
 * lx, ly: barycentric coordinates of x in tau and y in sigma (original local
 * vertex numbering); cc[a][b] = curl phi_a(tau) . curl phi_b(sigma);
 * nn = n_tau . n_sigma. */
static void accumulate(double blk[NOPS][3][3], double w, const double* lx, const double* ly,
                       const kern_vals* kv, double cc[3][3], double nn, double kappa) {
    double k2 = kappa * kappa;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double ll = lx[a] * ly[b];
            blk[0][a][b] += w * kv->gl * ll;
            blk[1][a][b] += w * kv->kl * ll;
            blk[2][a][b] += w * kv->gl * cc[a][b];
            blk[3][a][b] += w * kv->gy * ll;
            blk[4][a][b] += w * kv->ky * ll;
            blk[5][a][b] += w * kv->gy * (cc[a][b] + k2 * nn * ll);
        }
}

/* curl_G phi_a = -e_a / (2|tau|) on a flat triangle (e_a the edge opposite a). */
static void curl_products(const tri_geom* t, const tri_geom* s, double cc[3][3]) {
    double f = 1.0 / (4.0 * t->area * s->area);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) cc[a][b] = f * dot3(t->e[a], s->e[b]);
}

/* Regular pair: the same triangle rule on both triangles.
 * rule: nq points as barycentric triples (l0,l1,l2) and weights summing to 1. */
static void far_pair(const tri_geom* t, const tri_geom* s, int nq, const double* rl,
                     const double* rw, double kappa, double blk[NOPS][3][3]) {
    double cc[3][3];
    curl_products(t, s, cc);
    double nn = dot3(t->n, s->n);
    for (int i = 0; i < nq; ++i) {
        const double* lx = rl + 3 * i;
        double x[3];
        for (int k = 0; k < 3; ++k)
            x[k] = lx[0] * t->p[0][k] + lx[1] * t->p[1][k] + lx[2] * t->p[2][k];
        for (int j = 0; j < nq; ++j) {
            const double* ly = rl + 3 * j;
            double y[3];
            for (int k = 0; k < 3; ++k)
                y[k] = ly[0] * s->p[0][k] + ly[1] * s->p[1][k] + ly[2] * s->p[2][k];
            kern_vals kv = kernels(x, y, s->n, kappa);
            double w = rw[i] * t->area * rw[j] * s->area;
            accumulate(blk, w, lx, ly, &kv, cc, nn, kappa);
        }
    }
}

/* Point of the reordered reference triangle and its barycentrics in the
 * triangle's original numbering. perm[k] = original local index of the k-th
 * reordered vertex. */
static void ref_point(const tri_geom* g, const int* perm, double s, double t, double* x, double* lam) {
    double mu[3] = {1.0 - s, s - t, t};
    for (int k = 0; k < 3; ++k) lam[perm[k]] = mu[k];
    for (int k = 0; k < 3; ++k)
        x[k] = lam[0] * g->p[0][k] + lam[1] * g->p[1][k] + lam[2] * g->p[2][k];
}

/* Sauter-Schwab regions. Each fills (sx,tx),(sy,ty) and returns the region
 * Jacobian for the cube point (xi, e1, e2, e3). */
typedef double (*ss_map)(double xi, double e1, double e2, double e3, double* X, double* Y);

/* coincident panels: |y^-x^| is proportional to xi*e1*e2 in every region */
static double coin1(double xi, double e1, double e2, double e3, double* X, double* Y) {
    X[0] = xi; X[1] = xi * (1.0 - e1 + e1 * e2);
    Y[0] = xi * (1.0 - e1 * e2 * e3); Y[1] = xi * (1.0 - e1);
    return xi * xi * xi * e1 * e1 * e2;
}
static double coin2(double xi, double e1, double e2, double e3, double* X, double* Y) {
    return coin1(xi, e1, e2, e3, Y, X);
}
static double coin3(double xi, double e1, double e2, double e3, double* X, double* Y) {
    X[0] = xi; X[1] = xi * e1 * (1.0 - e2 + e2 * e3);
    Y[0] = xi * (1.0 - e1 * e2); Y[1] = xi * e1 * (1.0 - e2);
    return xi * xi * xi * e1 * e1 * e2;
}
static double coin4(double xi, double e1, double e2, double e3, double* X, double* Y) {
    return coin3(xi, e1, e2, e3, Y, X);
}
static double coin5(double xi, double e1, double e2, double e3, double* X, double* Y) {
    X[0] = xi * (1.0 - e1 * e2 * e3); X[1] = xi * e1 * (1.0 - e2 * e3);
    Y[0] = xi; Y[1] = xi * e1 * (1.0 - e2);
    return xi * xi * xi * e1 * e1 * e2;
}
static double coin6(double xi, double e1, double e2, double e3, double* X, double* Y) {
    return coin5(xi, e1, e2, e3, Y, X);
}

/* edge-adjacent panels: the common edge is t = 0 in both, x^ = y^ = (s, 0).
 * Derivation: write x^ = (s1, s1 w1), y^ = (s2, s2 w2) (Duffy square, measure
 * s1 s2). On s2 <= s1 put s1 = xi, s2 = xi (1 - h): measure xi^3 (1 - h), and
 * the singular set is the corner h = w1 = w2 = 0, where |x - y| is of the
 * order xi (h + w1 + w2). Split that cube by its largest coordinate (radial
 * variable e1, the other two scaled by it, Jacobian e1^2). The mirror half
 * s1 <= s2 swaps x^ and y^. Six regions in all. */
static double edge1(double xi, double e1, double e2, double e3, double* X, double* Y) {
    double s2 = xi * (1.0 - e1);                   /* h = e1 largest */
    X[0] = xi; X[1] = xi * e1 * e2;
    Y[0] = s2; Y[1] = s2 * e1 * e3;
    return xi * xi * xi * (1.0 - e1) * e1 * e1;
}
static double edge2(double xi, double e1, double e2, double e3, double* X, double* Y) {
    double s2 = xi * (1.0 - e1 * e2);              /* w1 = e1 largest */
    X[0] = xi; X[1] = xi * e1;
    Y[0] = s2; Y[1] = s2 * e1 * e3;
    return xi * xi * xi * (1.0 - e1 * e2) * e1 * e1;
}
static double edge3(double xi, double e1, double e2, double e3, double* X, double* Y) {
    double s2 = xi * (1.0 - e1 * e2);              /* w2 = e1 largest */
    X[0] = xi; X[1] = xi * e1 * e3;
    Y[0] = s2; Y[1] = s2 * e1;
    return xi * xi * xi * (1.0 - e1 * e2) * e1 * e1;
}
static double edge4(double xi, double e1, double e2, double e3, double* X, double* Y) {
    return edge1(xi, e1, e2, e3, Y, X);
}
static double edge5(double xi, double e1, double e2, double e3, double* X, double* Y) {
    return edge2(xi, e1, e2, e3, Y, X);
}
static double edge6(double xi, double e1, double e2, double e3, double* X, double* Y) {
    return edge3(xi, e1, e2, e3, Y, X);
}

/* vertex-adjacent panels: the common vertex is (0,0) in both */
static double vert1(double xi, double e1, double e2, double e3, double* X, double* Y) {
    X[0] = xi; X[1] = xi * e1;
    Y[0] = xi * e2; Y[1] = xi * e2 * e3;
    return xi * xi * xi * e2;
}
static double vert2(double xi, double e1, double e2, double e3, double* X, double* Y) {
    return vert1(xi, e1, e2, e3, Y, X);
}

static const ss_map COIN[6] = {coin1, coin2, coin3, coin4, coin5, coin6};
static const ss_map EDGE[6] = {edge1, edge2, edge3, edge4, edge5, edge6};
static const ss_map VERT[2] = {vert1, vert2};

/* Singular pair by the Sauter-Schwab regions. */
static void singular_pair(const tri_geom* t, const int* pt, const tri_geom* s, const int* ps,
                          const ss_map* maps, int nmaps, int ng, const double* gx,
                          const double* gw, double kappa, double blk[NOPS][3][3]) {
    double cc[3][3];
    curl_products(t, s, cc);
    double nn = dot3(t->n, s->n);
    double jac = (2.0 * t->area) * (2.0 * s->area);
    for (int m = 0; m < nmaps; ++m)
        for (int i0 = 0; i0 < ng; ++i0)
            for (int i1 = 0; i1 < ng; ++i1)
                for (int i2 = 0; i2 < ng; ++i2)
                    for (int i3 = 0; i3 < ng; ++i3) {
                        double X[2], Y[2];
                        double rj = maps[m](gx[i0], gx[i1], gx[i2], gx[i3], X, Y);
                        double w = gw[i0] * gw[i1] * gw[i2] * gw[i3] * rj * jac;
                        double x[3], y[3], lx[3], ly[3];
                        ref_point(t, pt, X[0], X[1], x, lx);
                        ref_point(s, ps, Y[0], Y[1], y, ly);
                        kern_vals kv = kernels(x, y, s->n, kappa);
                        accumulate(blk, w, lx, ly, &kv, cc, nn, kappa);
                    }
}

/* The distance band of the quadrature plan: the finer rule used on pairs that
 * share no vertex but lie closer than eta times the sum of their radii. */
typedef struct {
    double eta;         /* 0: no band */
    int nq;
    const double* rl;
    const double* rw;
} band_rule;

/* centroid and radius (largest centroid-vertex distance) of a triangle */
static void centroid_radius(const tri_geom* g, double* c, double* rho) {
    for (int k = 0; k < 3; ++k) c[k] = (g->p[0][k] + g->p[1][k] + g->p[2][k]) / 3.0;
    double r2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double d[3];
        sub3(g->p[a], c, d);
        double q = dot3(d, d);
        if (q > r2) r2 = q;
    }
    *rho = sqrt(r2);
}

static int in_band(const tri_geom* t, const tri_geom* s, double eta) {
    double ct[3], cs[3], rt, rs, d[3];
    centroid_radius(t, ct, &rt);
    centroid_radius(s, cs, &rs);
    sub3(ct, cs, d);
    double lim = eta * (rt + rs);
    return dot3(d, d) < lim * lim;
}

/* Local blocks of one triangle pair (test tau = tri ti, trial sigma = tri tj). */
static void pair_blocks(const double* verts, const int32_t* tris, int64_t ti, int64_t tj,
                        int nq, const double* rl, const double* rw, const int* ng, const double* gx,
                        const double* gw, double kappa, const band_rule* band, double blk[NOPS][3][3]) {
    memset(blk, 0, sizeof(double) * NOPS * 9);
    const int32_t* A = tris + 3 * ti;
    const int32_t* B = tris + 3 * tj;
    tri_geom t, s;
    make_geom(verts, A, &t);
    make_geom(verts, B, &s);
    /* shared vertices: (local index in tau, local index in sigma) */
    int sa[3], sb[3], ns = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (A[a] == B[b]) { sa[ns] = a; sb[ns] = b; ++ns; }
    if (ns == 0) {
        if (band && band->eta > 0.0 && in_band(&t, &s, band->eta))
            far_pair(&t, &s, band->nq, band->rl, band->rw, kappa, blk);
        else
            far_pair(&t, &s, nq, rl, rw, kappa, blk);
    } else if (ns == 3) {
        int id[3] = {0, 1, 2};
        singular_pair(&t, id, &s, id, COIN, 6, ng[0], gx, gw, kappa, blk);
    } else if (ns == 2) {
        /* reorder both so that the shared edge runs Q0 -> Q1 with the same
         * orientation in both parameterisations: from its lower to its higher
         * global vertex index, so that the rule of (sigma, tau) is the rule of
         * (tau, sigma) with the two roles exchanged */
        int k0 = A[sa[0]] < A[sa[1]] ? 0 : 1, k1 = 1 - k0;
        int pt[3] = {sa[k0], sa[k1], 3 - sa[0] - sa[1]};
        int ps[3] = {sb[k0], sb[k1], 3 - sb[0] - sb[1]};
        singular_pair(&t, pt, &s, ps, EDGE, 6, ng[1], gx + ng[0], gw + ng[0], kappa, blk);
    } else {
        int pt[3] = {sa[0], (sa[0] + 1) % 3, (sa[0] + 2) % 3};
        int ps[3] = {sb[0], (sb[0] + 1) % 3, (sb[0] + 2) % 3};
        singular_pair(&t, pt, &s, ps, VERT, 2, ng[2], gx + ng[0] + ng[1], gw + ng[0] + ng[1], kappa, blk);
    }
}

/* Exposed for unit tests: the six local blocks of one pair, [6][3][3]. */
int oracle_pair_blocks(const double* verts, const int32_t* tris, int64_t ti, int64_t tj, int nq,
                       const double* rl, const double* rw, const int* ng, const double* gx,
                       const double* gw, double kappa, double band_eta, int nbq, const double* brl,
                       const double* brw, double* out) {
    double blk[NOPS][3][3];
    band_rule band = {band_eta, nbq, brl, brw};
    pair_blocks(verts, tris, ti, tj, nq, rl, rw, ng, gx, gw, kappa, &band, blk);
    memcpy(out, blk, sizeof(blk));
    return 0;
}

/* Greedy colouring of triangles: no two triangles of one colour share a vertex. */
static int colour_triangles(const int32_t* tris, int64_t nt, int64_t nv, int* colour) {
    /* vertex -> bitmask of colours already used by its triangles (<= 64 colours) */
    uint64_t* used = (uint64_t*)calloc((size_t)nv, sizeof(uint64_t));
    if (!used) return -1;
    int ncol = 0;
    for (int64_t t = 0; t < nt; ++t) {
        uint64_t m = used[tris[3 * t]] | used[tris[3 * t + 1]] | used[tris[3 * t + 2]];
        int c = 0;
        while (c < 64 && (m >> c) & 1u) ++c;
        if (c == 64) { free(used); return -1; }
        colour[t] = c;
        if (c + 1 > ncol) ncol = c + 1;
        for (int a = 0; a < 3; ++a) used[tris[3 * t + a]] |= (uint64_t)1 << c;
    }
    free(used);
    return ncol;
}

/* Dense assembly. out: NOPS matrices of nv*nv doubles (row = test vertex),
 * plus the mass matrix mass[nv*nv]. Matrices must be zeroed by the caller. */
int oracle_assemble_dense(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                          int nq, const double* rl, const double* rw, const int* ng, const double* gx,
                          const double* gw, double kappa, double band_eta, int nbq, const double* brl,
                          const double* brw, int nthreads, double* VL, double* KL,
                          double* DL, double* VY, double* KY, double* DY, double* mass) {
    double* mats[NOPS] = {VL, KL, DL, VY, KY, DY};
    band_rule band = {band_eta, nbq, brl, brw};
    int* colour = (int*)malloc(sizeof(int) * (size_t)(nt > 0 ? nt : 1));
    if (!colour) return -1;
    int ncol = colour_triangles(tris, nt, nv, colour);
    if (ncol < 0) { free(colour); return -2; }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    for (int c = 0; c < ncol; ++c) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t ti = 0; ti < nt; ++ti) {
            if (colour[ti] != c) continue;
            const int32_t* A = tris + 3 * ti;
            for (int64_t tj = 0; tj < nt; ++tj) {
                double blk[NOPS][3][3];
                pair_blocks(verts, tris, ti, tj, nq, rl, rw, ng, gx, gw, kappa, &band, blk);
                const int32_t* B = tris + 3 * tj;
                for (int o = 0; o < NOPS; ++o)
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            mats[o][(int64_t)A[a] * nv + B[b]] += blk[o][a][b];
            }
            /* exact P1 mass matrix of tau: |tau|/12 [[2,1,1],[1,2,1],[1,1,2]] */
            tri_geom g;
            make_geom(verts, A, &g);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    mass[(int64_t)A[a] * nv + A[b]] += g.area / 12.0 * (a == b ? 2.0 : 1.0);
        }
    }
    free(colour);
    return ncol;
}

/* Row sample of the dense assembly: rows[r] is a test vertex; out matrices are
 * nrows*nv (row r of each), zeroed by the caller. Rows are independent, so
 * they are processed in parallel without any shared writes. */
int oracle_assemble_rows(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                         const int64_t* rows, int64_t nrows, int nq, const double* rl,
                         const double* rw, const int* ng, const double* gx, const double* gw,
                         double kappa, double band_eta, int nbq, const double* brl, const double* brw,
                         int nthreads, double* VL, double* KL, double* DL,
                         double* VY, double* KY, double* DY, double* mass) {
    double* mats[NOPS] = {VL, KL, DL, VY, KY, DY};
    band_rule band = {band_eta, nbq, brl, brw};
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        for (int64_t ti = 0; ti < nt; ++ti) {
            const int32_t* A = tris + 3 * ti;
            int a = -1;
            for (int k = 0; k < 3; ++k)
                if (A[k] == i) a = k;
            if (a < 0) continue;
            for (int64_t tj = 0; tj < nt; ++tj) {
                double blk[NOPS][3][3];
                pair_blocks(verts, tris, ti, tj, nq, rl, rw, ng, gx, gw, kappa, &band, blk);
                const int32_t* B = tris + 3 * tj;
                for (int o = 0; o < NOPS; ++o)
                    for (int b = 0; b < 3; ++b) mats[o][r * nv + B[b]] += blk[o][a][b];
            }
            tri_geom g;
            make_geom(verts, A, &g);
            for (int b = 0; b < 3; ++b)
                mass[r * nv + A[b]] += g.area / 12.0 * (a == b ? 2.0 : 1.0);
        }
    }
    return 0;
}

/* Source projections tested against the P1 basis (paper, "sources"):
 *   bD_i = int phi_i phi_D,  phi_D(x) = sum_j q_j / (4 pi eps_int |x - x_j|)
 *   bN_i = int phi_i phi_N,  phi_N(x) = -sum_j q_j (x - x_j).n_x / (4 pi eps_int |x - x_j|^3)
 * by the triangle rule on every triangle. Serial loop over triangles. */
int oracle_rhs(const double* verts, int64_t nv, const int32_t* tris, int64_t nt, int nq,
               const double* rl, const double* rw, const double* xq, const double* q, int64_t n_q,
               double eps_int, double* bD, double* bN) {
    memset(bD, 0, sizeof(double) * (size_t)nv);
    memset(bN, 0, sizeof(double) * (size_t)nv);
    for (int64_t ti = 0; ti < nt; ++ti) {
        tri_geom g;
        make_geom(verts, tris + 3 * ti, &g);
        for (int k = 0; k < nq; ++k) {
            const double* l = rl + 3 * k;
            double x[3];
            for (int c = 0; c < 3; ++c) x[c] = l[0] * g.p[0][c] + l[1] * g.p[1][c] + l[2] * g.p[2][c];
            double pd = 0.0, pn = 0.0;
            for (int64_t j = 0; j < n_q; ++j) {
                double d[3];
                sub3(x, xq + 3 * j, d);
                double r = sqrt(dot3(d, d));
                pd += q[j] / (4.0 * PI * eps_int * r);
                pn -= q[j] * dot3(d, g.n) / (4.0 * PI * eps_int * r * r * r);
            }
            double w = rw[k] * g.area;
            for (int a = 0; a < 3; ++a) {
                bD[tris[3 * ti + a]] += w * l[a] * pd;
                bN[tris[3 * ti + a]] += w * l[a] * pn;
            }
        }
    }
    return 0;
}

/* Reaction potential at the charges from interior traces (u = Dirichlet,
 * v = Neumann, P1 coefficients), paper eq. for phi_reac in boundary form:
 *   phi_reac(x_j) = int G_int(x_j,y) v(y) dy - int dG_int/dn_y(x_j,y) u(y) dy
 * by the triangle rule. Serial loops. */
int oracle_reaction_potential(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                              int nq, const double* rl, const double* rw, const double* u,
                              const double* v, const double* xq, int64_t n_q, double* phi) {
    (void)nv;
    for (int64_t j = 0; j < n_q; ++j) phi[j] = 0.0;
    for (int64_t ti = 0; ti < nt; ++ti) {
        tri_geom g;
        const int32_t* A = tris + 3 * ti;
        make_geom(verts, A, &g);
        for (int k = 0; k < nq; ++k) {
            const double* l = rl + 3 * k;
            double y[3];
            for (int c = 0; c < 3; ++c) y[c] = l[0] * g.p[0][c] + l[1] * g.p[1][c] + l[2] * g.p[2][c];
            double uy = l[0] * u[A[0]] + l[1] * u[A[1]] + l[2] * u[A[2]];
            double vy = l[0] * v[A[0]] + l[1] * v[A[1]] + l[2] * v[A[2]];
            double w = rw[k] * g.area;
            for (int64_t j = 0; j < n_q; ++j) {
                kern_vals kv = kernels(xq + 3 * j, y, g.n, 0.0);
                phi[j] += w * (kv.gl * vy - kv.kl * uy);
            }
        }
    }
    return 0;
}

/* Number of ordered triangle pairs (ti, tj), ti != tj, that share no vertex and
 * lie in the distance band of eta (in_band): the pairs on which a banded plan
 * uses the band rule instead of the far rule. A plain loop over all pairs. */
int64_t oracle_band_pair_count(const double* verts, const int32_t* tris, int64_t nt, double eta, int nthreads) {
    int64_t count = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : count)
    for (int64_t ti = 0; ti < nt; ++ti) {
        tri_geom t;
        make_geom(verts, tris + 3 * ti, &t);
        for (int64_t tj = 0; tj < nt; ++tj) {
            if (tj == ti) continue;
            const int32_t* A = tris + 3 * ti;
            const int32_t* B = tris + 3 * tj;
            int shared = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) shared |= A[a] == B[b];
            if (shared) continue;
            tri_geom s;
            make_geom(verts, B, &s);
            count += in_band(&t, &s, eta);
        }
    }
    return count;
}

/* Exposed for unit tests of the singular maps: integral over [0,1]^4 of the
 * region Jacobian times s_x^a t_x^b s_y^c t_y^d, summed over the regions of
 * one kind (0 = coincident, 1 = edge, 2 = vertex). For correct maps this is
 * the product of the two reference-triangle moments. */
double oracle_ss_moment(int kind, int ng, const double* gx, const double* gw, int a, int b, int c,
                        int d) {
    const ss_map* maps = kind == 0 ? COIN : (kind == 1 ? EDGE : VERT);
    int nmaps = kind == 0 ? 6 : (kind == 1 ? 6 : 2);
    double sum = 0.0;
    for (int m = 0; m < nmaps; ++m)
        for (int i0 = 0; i0 < ng; ++i0)
            for (int i1 = 0; i1 < ng; ++i1)
                for (int i2 = 0; i2 < ng; ++i2)
                    for (int i3 = 0; i3 < ng; ++i3) {
                        double X[2], Y[2];
                        double rj = maps[m](gx[i0], gx[i1], gx[i2], gx[i3], X, Y);
                        sum += gw[i0] * gw[i1] * gw[i2] * gw[i3] * rj * pow(X[0], a) *
                               pow(X[1], b) * pow(Y[0], c) * pow(Y[1], d);
                    }
    return sum;
}
