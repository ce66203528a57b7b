// a2: FP64 near field. For every ordered pair of triangles sharing a vertex,
// the local 3x3 Galerkin blocks of V, K, D (Laplace and Yukawa) by a
// regularised [0,1]^4 rule (maps in the manner of Sauter and Schwab, with a
// Gauss-Legendre product rule), minus the same blocks by the far rule that the
// pair kernel applies to every pair, summed into the vertex-pair CSR. The full
// (regularised) diagonals are kept for the block-diagonal preconditioner.
//
// Operators (paper eq. layer_potentials, weak forms on P1):
//   V_ab = int int l_a(x) G(x,y) l_b(y)       K_ab = int int l_a(x) dG/dn_y l_b(y)
//   D_ab = int int G [curl l_a . curl l_b + kappa^2 n_x.n_y l_a l_b]  (hypersingular,
//          integrated by parts; curl l_a = -e_a / (2|tau|), e_a the edge opposite a)
// with G_int = 1/(4 pi r), G_ext = exp(-kappa r)/(4 pi r).
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "internal.h"

namespace pb {

struct Gauss {
    double x[12];
    double w[12];
    int n;
};

// Gauss-Legendre nodes on [0,1] by Newton's method on P_n (three-term
// recurrence for P_n, derivative from P_n and P_{n-1}).
static Gauss gauss01(int n) {
    Gauss g;
    g.n = n;
    for (int i = 0; i < n; ++i) {
        double x = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = x; p0 = 1.0; }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        // recompute the derivative at the converged node for the weight
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) { p1 = x; p0 = 1.0; }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        double w = 2.0 / ((1.0 - x * x) * dp * dp);
        g.x[i] = 0.5 * (1.0 - x);  // ascending on [0,1]
        g.w[i] = 0.5 * w;
    }
    return g;
}

// One regularised cube point -> reference points (sx,tx) in tau and (sy,ty)
// in sigma on {0 <= t <= s <= 1}, returning the region Jacobian.
// kind 0: coincident (6 regions), 1: common edge t = 0 (6), 2: common vertex (0,0) (2).
__device__ __forceinline__ double ss_map(int kind, int reg, double xi, double e1, double e2, double e3,
                                         double& sx, double& tx, double& sy, double& ty) {
    double a0, a1, b0, b1, jac;
    int base = reg;
    bool swap = false;
    if (kind == 2) {
        swap = reg == 1;
        a0 = xi; a1 = xi * e1;
        b0 = xi * e2; b1 = xi * e2 * e3;
        jac = xi * xi * xi * e2;
    } else {
        if (reg >= 3) { base = reg - 3; swap = true; }
        if (kind == 0) {
            jac = xi * xi * xi * e1 * e1 * e2;
            if (base == 0) {
                a0 = xi; a1 = xi * (1.0 - e1 + e1 * e2);
                b0 = xi * (1.0 - e1 * e2 * e3); b1 = xi * (1.0 - e1);
            } else if (base == 1) {
                a0 = xi; a1 = xi * e1 * (1.0 - e2 + e2 * e3);
                b0 = xi * (1.0 - e1 * e2); b1 = xi * e1 * (1.0 - e2);
            } else {
                a0 = xi * (1.0 - e1 * e2 * e3); a1 = xi * e1 * (1.0 - e2 * e3);
                b0 = xi; b1 = xi * e1 * (1.0 - e2);
            }
        } else {
            // x^ = (s1, s1 w1), y^ = (s2, s2 w2), s1 = xi, s2 = xi (1 - h); the
            // largest of (h, w1, w2) is e1 and the other two are e1 times (e2, e3)
            double h, w1, w2;
            if (base == 0) { h = e1; w1 = e1 * e2; w2 = e1 * e3; }
            else if (base == 1) { w1 = e1; h = e1 * e2; w2 = e1 * e3; }
            else { w2 = e1; h = e1 * e2; w1 = e1 * e3; }
            double s2 = xi * (1.0 - h);
            a0 = xi; a1 = xi * w1;
            b0 = s2; b1 = s2 * w2;
            jac = xi * xi * xi * (1.0 - h) * e1 * e1;
        }
    }
    if (swap) { sx = b0; tx = b1; sy = a0; ty = a1; }
    else { sx = a0; tx = a1; sy = b0; ty = b1; }
    return jac;
}

// The regularised rule of the coincident pairs does not depend on the pair:
// every (region, Gauss index) point of regions 0..2 of the coincident map, its
// reference points in both copies of the triangle and its weight (Gauss
// weights times the region Jacobian), computed once per build. Structure of
// arrays over the entries.
struct SSTable {
    const double* sx;
    const double* tx;
    const double* sy;
    const double* ty;
    const double* w;
    // w times the monomials (s', t', s, s s', s t', t, t s', t t') of the
    // entry's frame coordinates: mono[c * n + e]
    const double* mono;
    int n;       // entries in all (3 n^4)
};
constexpr int SS_TABLE_ARRAYS = 13;  // sx, tx, sy, ty, w and the eight weighted monomials

__global__ void k_ss_table(Gauss gq, int n, double* __restrict__ tab) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int q = gq.n, n4 = q * q * q * q;
    const int reg = e / n4, r = e - reg * n4;
    const int i0 = r / (q * q * q), i1 = (r / (q * q)) % q, i2 = (r / q) % q, i3 = r % q;
    double sx, tx, sy, ty;
    const double jac = ss_map(0, reg, gq.x[i0], gq.x[i1], gq.x[i2], gq.x[i3], sx, tx, sy, ty);
    tab[e] = sx;
    tab[n + e] = tx;
    tab[2 * n + e] = sy;
    tab[3 * n + e] = ty;
    const double w = gq.w[i0] * gq.w[i1] * gq.w[i2] * gq.w[i3] * jac;
    tab[4 * n + e] = w;
    const double ws = w * sx, wt = w * tx;
    const double mono[8] = {w * sy, w * ty, ws, ws * sy, ws * ty, wt, wt * sy, wt * ty};
    for (int c = 0; c < 8; ++c) tab[(5 + c) * n + e] = mono[c];
}

// Outer points of the edge (kind 1, 6 regions) and vertex (kind 2, 2 regions)
// maps: one entry per (region, xi, eta1, eta2). In both maps the innermost
// Gauss variable eta3 enters a single coordinate, the second one (t) of one
// frame, and linearly, while the region Jacobian does not involve it; so
// over the eta3 points of an entry x - y = D0 + eta3 D1 and every weighted
// monomial is affine in eta3. A pair's kernel sums then take two partial sums
// per kernel over eta3 (sum w3 g, sum w3 eta3 g) and expand them into the
// nine moments once per entry. Per entry (array c at v[c * n + e]):
//   0..3  sa, ta, sa', ta': the frame coordinates at eta3 = 0 (x: s, t; y: s', t')
//   4, 5  tb, tb': the slopes of t and t' in eta3 (one of them is zero)
//   6..14 c0[3 alpha + beta] = W P_alpha Q_beta, P = (1, sa, ta), Q = (1, sa', ta'),
//         W = the Gauss weights of xi, eta1, eta2 times the Jacobian
//   15..19 the eta3-slope coefficients of the moments that change with eta3:
//         (0,2) W tb', (1,2) W sa tb', (2,0) W tb, (2,1) W tb sa', (2,2) W (ta tb' + tb ta')
// followed by the eta3 Gauss nodes and weights (2 n doubles).
// One table per class (edge or vertex), each with its own Gauss rule.
struct SSOuter {
    const double* v;
    int n;        // entries (regions x nss^3)
    int nss;      // Gauss points per dimension
    int nreg;     // regions of the map: 6 (edge) or 2 (vertex)
};
constexpr int SS_OUTER_ARRAYS = 20;

__global__ void k_ss_outer(Gauss gq, int kind, int n, double* __restrict__ tab) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int q = gq.n, n3 = q * q * q;
    if (e < 2 * q) {  // the eta3 rule after the entries
        tab[SS_OUTER_ARRAYS * n + e] = e < q ? gq.x[e] : gq.w[e - q];
    }
    if (e >= n) return;
    const int reg = e / n3, r = e - reg * n3;
    const int i0 = r / (q * q), i1 = (r / q) % q, i2 = r % q;
    double sx0, tx0, sy0, ty0, sx1, tx1, sy1, ty1;
    const double jac = ss_map(kind, reg, gq.x[i0], gq.x[i1], gq.x[i2], 0.0, sx0, tx0, sy0, ty0);
    const double jac1 = ss_map(kind, reg, gq.x[i0], gq.x[i1], gq.x[i2], 1.0, sx1, tx1, sy1, ty1);
    const double tb = tx1 - tx0, tb2 = ty1 - ty0;
    const double W = gq.w[i0] * gq.w[i1] * gq.w[i2] * jac;
    // the structure the factorisation relies on: s, s' and the Jacobian free of eta3
    const bool ok = sx1 == sx0 && sy1 == sy0 && jac1 == jac;
    const double P[3] = {1.0, sx0, tx0}, Q[3] = {1.0, sy0, ty0};
    double v[SS_OUTER_ARRAYS] = {sx0, tx0, sy0, ty0, tb, tb2};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) v[6 + 3 * a + b] = ok ? W * P[a] * Q[b] : __longlong_as_double(0x7ff8000000000000LL);
    v[15] = W * tb2;
    v[16] = W * sx0 * tb2;
    v[17] = W * tb;
    v[18] = W * tb * sy0;
    v[19] = W * (tx0 * tb2 + tb * ty0);
    for (int c = 0; c < SS_OUTER_ARRAYS; ++c) tab[c * n + e] = v[c];
}

// Geometry of one triangle in the reordered frame of its singular map:
// Q0, E1 = Q1 - Q0, E2 = Q2 - Q1 (x(s,t) = Q0 + s E1 + t E2), the inverse
// permutation (original corner -> reordered), normal and area. Kept in shared
// memory per warp: the lanes read it by broadcast.
struct TriFrame {
    double q0[3], e1[3], e2[3];
    double n[3];
    double area;
    int inv[3];  // reordered index of original corner a
};

__device__ void make_frame(const double* verts, const int32_t* tris, const double* tgeo, int t, int perm,
                           TriFrame& f) {
    double p[3][3];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) p[a][k] = verts[3 * (int64_t)tris[3 * (int64_t)t + a] + k];
    int o[3] = {perm & 3, (perm >> 2) & 3, (perm >> 4) & 3};  // original corner of reordered k
    for (int k = 0; k < 3; ++k) {
        f.q0[k] = p[o[0]][k];
        f.e1[k] = p[o[1]][k] - p[o[0]][k];
        f.e2[k] = p[o[2]][k] - p[o[1]][k];
        f.n[k] = tgeo[16 * (int64_t)t + k];
    }
    f.area = tgeo[16 * (int64_t)t + 3];
    for (int k = 0; k < 3; ++k) f.inv[o[k]] = k;
}

// original corner a of the triangle
__device__ __forceinline__ double corner(const TriFrame& f, int a, int k) {
    int r = f.inv[a];
    return f.q0[k] + (r >= 1 ? f.e1[k] : 0.0) + (r >= 2 ? f.e2[k] : 0.0);
}

// e^x for x <= 0 (the Yukawa factor e^{-kappa r}) by the table-driven method
// of Tang (ACM Trans. Math. Software 15(2), 1989): x = (32 m + j) ln2/32 + r
// with |r| <= ln2/64, and e^x = 2^m 2^{j/32} e^r, with 2^{j/32} from a table
// (correctly rounded doubles) and e^r its Taylor polynomial of degree 6
// (remainder below 2e-18). The reduction subtracts n ln2/32 in two parts, the
// first with 37 significant bits so that n times it is exact for |n| < 2^15.
// Arguments below -700 give 0 (the exact value is below 1e-304).
__device__ const double g_exp2_32[32] = {
    0x1.0000000000000p+0, 0x1.059b0d3158574p+0, 0x1.0b5586cf9890fp+0, 0x1.11301d0125b51p+0,
    0x1.172b83c7d517bp+0, 0x1.1d4873168b9aap+0, 0x1.2387a6e756238p+0, 0x1.29e9df51fdee1p+0,
    0x1.306fe0a31b715p+0, 0x1.371a7373aa9cbp+0, 0x1.3dea64c123422p+0, 0x1.44e086061892dp+0,
    0x1.4bfdad5362a27p+0, 0x1.5342b569d4f82p+0, 0x1.5ab07dd485429p+0, 0x1.6247eb03a5585p+0,
    0x1.6a09e667f3bcdp+0, 0x1.71f75e8ec5f74p+0, 0x1.7a11473eb0187p+0, 0x1.82589994cce13p+0,
    0x1.8ace5422aa0dbp+0, 0x1.93737b0cdc5e5p+0, 0x1.9c49182a3f090p+0, 0x1.a5503b23e255dp+0,
    0x1.ae89f995ad3adp+0, 0x1.b7f76f2fb5e47p+0, 0x1.c199bdd85529cp+0, 0x1.cb720dcef9069p+0,
    0x1.d5818dcfba487p+0, 0x1.dfc97337b9b5fp+0, 0x1.ea4afa2a490dap+0, 0x1.f50765b6e4540p+0};

__device__ __forceinline__ double exp_nonpos(double x) {
    const double shifter = 0x1.8p52;  // adding it rounds to an integer held in the low mantissa bits
    const double tn = __fma_rn(x, 0x1.71547652b82fep+5, shifter);  // x 32/ln2, rounded
    const int n = __double2loint(tn);
    const double nd = __dsub_rn(tn, shifter);
    const double r = __fma_rn(-nd, 0x1.cf79abc9e3b3ap-45, __fma_rn(-nd, 0x1.62e42fefa0000p-6, x));
    double q = 1.0 / 720.0;
    q = __fma_rn(q, r, 1.0 / 120.0);
    q = __fma_rn(q, r, 1.0 / 24.0);
    q = __fma_rn(q, r, 1.0 / 6.0);
    q = __fma_rn(q, r, 0.5);
    q = __fma_rn(q, r, 1.0);
    q = __fma_rn(q, r, 1.0);
    const double v = __ldg(g_exp2_32 + (n & 31)) * q;
    const long long bits = __double_as_longlong(v) + ((long long)(n >> 5) << 52);  // times 2^m
    return x < -700.0 ? 0.0 : __longlong_as_double(bits);
}

// Accumulators: SL[9], SY[9], KL[9], KY[9], sum w G_L, sum w G_Y (38); with
// the reversed pair also KTL[9], KTY[9] (56): the double-layer kernel with the
// normal of the first triangle, which is the K block of the reversed pair.
#define NACC_NEAR 38
#define NACC_SYM 56

template <bool SYM>
__device__ __forceinline__ void accum_point(double* acc, double w, const double* x, const double* y,
                                            const double* nx, const double* ny, const double* lx,
                                            const double* ly, double kappa) {
    const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
    const double rinv = rsqrt(r2);
    const double r = r2 * rinv;
    const double gl = rinv * 0.07957747154594767;  // 1 / (4 pi r)
    const double ek = exp_nonpos(-kappa * r);
    const double gy = ek * gl;
    const double fl = gl * rinv * rinv;            // 1 / (4 pi r^3)
    const double fy_over_fl = ek * (1.0 + kappa * r);
    const double dn = d0 * ny[0] + d1 * ny[1] + d2 * ny[2];
    const double kl = fl * dn;
    const double ky = kl * fy_over_fl;
    double ktl = 0.0, kty = 0.0;
    if (SYM) {
        const double dnx = -(d0 * nx[0] + d1 * nx[1] + d2 * nx[2]);  // (y - x).n_x
        ktl = fl * dnx;
        kty = ktl * fy_over_fl;
    }
    for (int a = 0; a < 3; ++a) {
        const double wa = w * lx[a];
        for (int b = 0; b < 3; ++b) {
            const double ll = wa * ly[b];
            acc[3 * a + b] += gl * ll;
            acc[9 + 3 * a + b] += gy * ll;
            acc[18 + 3 * a + b] += kl * ll;
            acc[27 + 3 * a + b] += ky * ll;
            if (SYM) {
                acc[38 + 3 * a + b] += ktl * ll;
                acc[47 + 3 * a + b] += kty * ll;
            }
        }
    }
    acc[36] += w * gl;
    acc[37] += w * gy;
}

// Regularised rules in the frames' own coordinates. A point of a frame is
// q0 + s e1 + t e2 and its corner basis values are mu = (1 - s, s - t, t) in the
// frame's corner order; so the quadrature sums are taken as moments in the
// monomial bases (1, s, t) x (1, s', t') and turned into the corner blocks once
// per pair (frame_to_corner). For an adjacent pair both frames start at the
// shared vertex, and d = x - y is formed from the frame vectors directly.
// mom[9 k + 3 alpha + beta], k = G_L, G_Y, K_L, K_Y (and with SYM the reversed
// pair's double layers K^T_L, K^T_Y).
// Kernel values at x - y = d for an adjacent pair: G_L, G_Y, the double layers
// K_L, K_Y with the second triangle's normal and (SYM) the reversed pair's with
// the first triangle's normal.
template <bool SYM>
__device__ __forceinline__ void adj_kernels(const double* d, const TriFrame& A, const TriFrame& B, double kappa,
                                            double* g) {
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double rinv = rsqrt(r2);
    const double r = r2 * rinv;
    const double gl = rinv * 0.07957747154594767;  // 1 / (4 pi r)
    const double ek = exp_nonpos(-kappa * r);
    const double fl = gl * rinv * rinv;  // 1 / (4 pi r^3)
    const double fy_over_fl = ek * (1.0 + kappa * r);
    const double kl = fl * (d[0] * B.n[0] + d[1] * B.n[1] + d[2] * B.n[2]);
    g[0] = gl;
    g[1] = ek * gl;
    g[2] = kl;
    g[3] = kl * fy_over_fl;
    if (SYM) {
        const double ktl = fl * -(d[0] * A.n[0] + d[1] * A.n[1] + d[2] * A.n[2]);  // (y - x).n_x
        g[4] = ktl;
        g[5] = ktl * fy_over_fl;
    }
}

// One outer entry (region, xi, eta1, eta2) of an edge- or vertex-adjacent pair:
// the NSS eta3 points summed per kernel into a0 = sum w3 g and a1 = sum w3 eta3 g,
// then expanded into the moments (nine per kernel from a0, five from a1).
// NSS = 0: the rule's size is read at run time.
template <bool SYM, int NSS>
__device__ __forceinline__ void accum_outer(double* mom, const SSOuter& tab, int e, const double* dq,
                                            const TriFrame& A, const TriFrame& B, double kappa, const double* x3,
                                            const double* w3) {
    constexpr int NK = SYM ? 6 : 4;
    const int n = tab.n;
    const double sa = tab.v[e], ta = tab.v[n + e], sa2 = tab.v[2 * n + e], ta2 = tab.v[3 * n + e];
    const double tb = tab.v[4 * n + e], tb2 = tab.v[5 * n + e];
    double D0[3], D1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        D0[k] = __fma_rn(-ta2, B.e2[k], __fma_rn(-sa2, B.e1[k], __fma_rn(ta, A.e2[k], __fma_rn(sa, A.e1[k], dq[k]))));
        D1[k] = __fma_rn(tb, A.e2[k], -tb2 * B.e2[k]);
    }
    double a0[NK], a1[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) a0[k] = a1[k] = 0.0;
    const int nss = NSS > 0 ? NSS : tab.nss;
#pragma unroll
    for (int j = 0; j < (NSS > 0 ? NSS : 12); ++j) {
        if (NSS == 0 && j >= nss) break;
        const double x = x3[j], w = w3[j], wx = w * x;
        double d[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) d[k] = __fma_rn(x, D1[k], D0[k]);
        double g[6];
        adj_kernels<SYM>(d, A, B, kappa, g);
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            a0[k] = __fma_rn(w, g[k], a0[k]);
            a1[k] = __fma_rn(wx, g[k], a1[k]);
        }
    }
    double c0[9], c1[5];
#pragma unroll
    for (int c = 0; c < 9; ++c) c0[c] = tab.v[(6 + c) * n + e];
#pragma unroll
    for (int c = 0; c < 5; ++c) c1[c] = tab.v[(15 + c) * n + e];
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        double* mk = mom + 9 * k;
#pragma unroll
        for (int c = 0; c < 9; ++c) mk[c] = __fma_rn(c0[c], a0[k], mk[c]);
        mk[2] = __fma_rn(c1[0], a1[k], mk[2]);
        mk[5] = __fma_rn(c1[1], a1[k], mk[5]);
        mk[6] = __fma_rn(c1[2], a1[k], mk[6]);
        mk[7] = __fma_rn(c1[3], a1[k], mk[7]);
        mk[8] = __fma_rn(c1[4], a1[k], mk[8]);
    }
}

// coincident pair: one frame, d = (s - s') e1 + (t - t') e2; k = G_L, G_Y
__device__ __forceinline__ void accum_coin_frame(double* mom, const SSTable& tab, int e, const TriFrame& A,
                                                 double kappa) {
    const double ds = tab.sx[e] - tab.sy[e], dt = tab.tx[e] - tab.ty[e];
    double d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = __fma_rn(dt, A.e2[k], ds * A.e1[k]);
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double rinv = rsqrt(r2);
    const double gl = rinv * 0.07957747154594767;  // 1 / (4 pi r)
    const double gy = exp_nonpos(-kappa * (r2 * rinv)) * gl;
    double m[9];
    m[0] = tab.w[e];
#pragma unroll
    for (int c = 0; c < 8; ++c) m[1 + c] = tab.mono[c * tab.n + e];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        mom[c] += gl * m[c];
        mom[9 + c] += gy * m[c];
    }
}

// moments of one kernel (mom[3 alpha + beta] over (1, s, t) x (1, s', t')) into
// its corner block out[3 a + b] = sum w g l_a(x) l_b(y)
__device__ __forceinline__ void frame_to_corner(const double* mom, const TriFrame& A, const TriFrame& B,
                                                double* out) {
    double R[3][3], U[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {  // mu_0 = 1 - s, mu_1 = s - t, mu_2 = t on the first frame
        R[0][b] = mom[b] - mom[3 + b];
        R[1][b] = mom[3 + b] - mom[6 + b];
        R[2][b] = mom[6 + b];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {  // and on the second
        U[a][0] = R[a][0] - R[a][1];
        U[a][1] = R[a][1] - R[a][2];
        U[a][2] = R[a][2];
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) out[3 * a + b] = U[A.inv[a]][B.inv[b]];
}

// One level of a warp reduce-scatter: a lane keeps half of its first 2H
// entries (the upper half when its bit o is set) and adds its partner's copy.
template <int H>
__device__ __forceinline__ void rs_level(double* v, int lane, int o) {
    const bool up = lane & o;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const double lo = v[i], hi = v[i + H];
        v[i] = (up ? hi : lo) + __shfl_xor_sync(0xffffffffu, up ? lo : hi, o);
    }
}

// Warp sums of v[0..NV) into every lane's v. A reduce-scatter over the five
// lane bits (offsets 16 .. 1, N the power of two with NV <= N <= 2 NV, entries
// past NV being zero) leaves lane L with the totals of entries [L N/32,
// (L + 1) N/32) after N/2 + N/4 + ... + N/32 additions, against 5 NV for a
// butterfly on every entry; the totals go through the warp's shared buffer
// (N doubles) back to all lanes. Fixed order: deterministic.
template <int NV, int N>
__device__ __forceinline__ void warp_allsum(double* v, int lane, double* buf) {
    static_assert(N >= 32 && (N & (N - 1)) == 0 && NV <= N && 2 * NV >= N, "reduce-scatter size");
    {
        constexpr int h = N / 2;
        const bool up = lane & 16;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const double lo = v[i], hi = i + h < NV ? v[i + h] : 0.0;
            v[i] = (up ? hi : lo) + __shfl_xor_sync(0xffffffffu, up ? lo : hi, 16);
        }
    }
    rs_level<N / 4>(v, lane, 8);
    rs_level<N / 8>(v, lane, 4);
    rs_level<N / 16>(v, lane, 2);
    rs_level<N / 32>(v, lane, 1);
    constexpr int K = N / 32;
#pragma unroll
    for (int j = 0; j < K; ++j) buf[lane * K + j] = v[j];
    __syncwarp();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = buf[k];
    __syncwarp();  // the buffer is free again
}


// Six 3x3 blocks (V_L, K_L, D_L, V_Y, K_Y, D_Y) of the pair (tau, sigma), or with
// rev = true of the reversed pair (sigma, tau): every block transposed and the
// double layer taken from the KT accumulators. Layout: out[6 (3a + b) + k] for
// corner a of the test triangle, corner b of the trial one and operator k, so
// that the six values one row-assembly lane reads are 48 contiguous bytes.
__device__ void expand_blocks(const double* acc, const TriFrame& A, const TriFrame& B, const double* tgeoA,
                              const double* tgeoB, double kappa, bool rev, double* out) {
    double nn = A.n[0] * B.n[0] + A.n[1] * B.n[1] + A.n[2] * B.n[2];
    double f = 1.0 / (4.0 * A.area * B.area);
    const int kL = rev ? 38 : 18, kY = rev ? 47 : 27;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const double* ea = tgeoA + 4 + 3 * a;
            const double* eb = tgeoB + 4 + 3 * b;
            double cc = f * (ea[0] * eb[0] + ea[1] * eb[1] + ea[2] * eb[2]);
            const int ab = 3 * a + b;
            const int o = rev ? 3 * b + a : ab;
            double* e = out + 6 * o;
            e[0] = acc[ab];
            e[1] = acc[kL + ab];
            e[2] = cc * acc[36];
            e[3] = acc[9 + ab];
            e[4] = acc[kY + ab];
            e[5] = cc * acc[37] + kappa * kappa * nn * acc[9 + ab];
        }
}

constexpr int NEAR_THREADS = 128;

// FP64 flops per quadrature point pair by formula count (a fused multiply-add
// counted as two). NEAR_FLOPS_SYM: one point pair with all six kernels and a
// direct accumulation into the 3x3 blocks (the far-rule pairs of an adjacent
// pair, accum_point). Kernel evaluation: d = x - y (24 when formed from frame
// vectors); r^2 (5), rsqrt, r, 1/(4 pi r), kappa r, exp, the Yukawa single
// layer (6), 1/r^3 (2), (1 + kappa r) and the Yukawa double-layer factor (3),
// d.n_y (5) and both double layers (2): 47; with the reversed pair's double
// layer, d.n_x (5) and its two kernels (2): 54. Accumulation: one FMA per
// kernel and block entry, 2 x 6 x 9 (108). Coincident pairs (moments from the
// rule's table of weighted monomials): d from (s - s', t - t') (11), r^2 to
// the Yukawa single layer (11); 2 x 2 x 9 (36).
constexpr double NEAR_FLOPS_SYM = 54 + 108;
constexpr double NEAR_FLOPS_COIN = 22 + 36;
// The factorised adjacent-pair sums (accum_outer): per quadrature point pair
// the kernel evaluation with d = D0 + eta3 D1 (3 FMA instead of 12: 36) and the
// two partial sums per kernel (2 x 6 FMA: 24); per outer entry D0 and D1
// (12 FMA, 3 FMA and 3 products: 33) and the moments (6 kernels x 14 FMA: 168).
constexpr double NEAR_FLOPS_ADJ_POINT = 36 + 24;
constexpr double NEAR_FLOPS_ADJ_OUTER = 33 + 168;

// One warp per listed pair. Writes ss[p][54] (regularised) and far[p][54] (far
// rule, identical points excluded); with SYM also the blocks of the reversed
// pair rev[p], whose rule is this one with the roles exchanged.
template <int MINB, bool SYM, int NSS>
__global__ void __launch_bounds__(NEAR_THREADS, MINB)
k_near_pairs(const double* __restrict__ verts, const int32_t* __restrict__ tris, const double* __restrict__ tgeo,
             const int4* __restrict__ pairs, const int32_t* __restrict__ list, int64_t nlist,
             const int32_t* __restrict__ rev, SSOuter tab, Rule rule, double kappa,
             double* __restrict__ ss_out, double* __restrict__ far_out) {
    constexpr int NA = SYM ? NACC_SYM : NACC_NEAR;
    constexpr int NM = SYM ? 54 : 36;  // frame moments
    __shared__ TriFrame frames[NEAR_THREADS / 32][2];
    __shared__ double red[NEAR_THREADS / 32][64];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t li = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (li >= nlist) return;  // whole warps leave together
    const int64_t p = list[li];
    const int4 pr = pairs[p];
    TriFrame& A = frames[wid][0];
    TriFrame& B = frames[wid][1];
    if (lane == 0) make_frame(verts, tris, tgeo, pr.x, pr.w & 63, A);
    if (lane == 1) make_frame(verts, tris, tgeo, pr.y, (pr.w >> 6) & 63, B);
    __syncwarp();
    const int nreg = tab.nreg;  // every pair of the list has the table's class
    const int e0 = 0;
    const int n3 = tab.nss * tab.nss * tab.nss;
    const double jac_ab = (2.0 * A.area) * (2.0 * B.area);
    const double dq[3] = {A.q0[0] - B.q0[0], A.q0[1] - B.q0[1], A.q0[2] - B.q0[2]};  // 0: the shared vertex
    // the eta3 rule, in registers for a fixed size
    double x3[NSS > 0 ? NSS : 1], w3[NSS > 0 ? NSS : 1];
    const double* rule3 = tab.v + (size_t)SS_OUTER_ARRAYS * tab.n;
    if (NSS > 0) {
#pragma unroll
        for (int j = 0; j < (NSS > 0 ? NSS : 1); ++j) {
            x3[j] = rule3[j];
            w3[j] = rule3[tab.nss + j];
        }
    }
    double acc[NA];
    {
        double mom[NM];
        for (int k = 0; k < NM; ++k) mom[k] = 0.0;
        for (int idx = lane; idx < nreg * n3; idx += 32)
            accum_outer<SYM, NSS>(mom, tab, e0 + idx, dq, A, B, kappa, NSS > 0 ? x3 : rule3,
                                  NSS > 0 ? w3 : rule3 + tab.nss);
        warp_allsum<NM, 64>(mom, lane, red[wid]);
        for (int k = 0; k < NM; ++k) mom[k] *= jac_ab;  // the pair's Jacobian, once
        // corner blocks in the accumulator layout of accum_point
        for (int k = 0; k < NM / 9; ++k) frame_to_corner(mom + 9 * k, A, B, acc + (k < 4 ? 9 * k : 38 + 9 * (k - 4)));
        acc[36] = mom[0];  // sum w G_L: the (1, 1) moment
        acc[37] = mom[9];
    }
    const double* gA = tgeo + 16 * (int64_t)pr.x;
    const double* gB = tgeo + 16 * (int64_t)pr.y;
    if (lane == 0) expand_blocks(acc, A, B, gA, gB, kappa, false, ss_out + 54 * p);
    if (SYM && lane == 1) expand_blocks(acc, A, B, gA, gB, kappa, true, ss_out + 54 * (int64_t)rev[p]);
    // far rule on the same pair (what the pair kernel adds for it)
    for (int k = 0; k < NA; ++k) acc[k] = 0.0;
    const int Q = rule.Q;
    for (int idx = lane; idx < Q * Q; idx += 32) {
        const int i = idx / Q, j = idx % Q;
        double x[3], y[3];
        for (int k = 0; k < 3; ++k) {
            x[k] = rule.l[i][0] * corner(A, 0, k) + rule.l[i][1] * corner(A, 1, k) + rule.l[i][2] * corner(A, 2, k);
            y[k] = rule.l[j][0] * corner(B, 0, k) + rule.l[j][1] * corner(B, 1, k) + rule.l[j][2] * corner(B, 2, k);
        }
        const double w = rule.w[i] * A.area * rule.w[j] * B.area;
        accum_point<SYM>(acc, w, x, y, A.n, B.n, rule.l[i], rule.l[j], kappa);
    }
    warp_allsum<NA, 64>(acc, lane, red[wid]);
    if (lane == 0) expand_blocks(acc, A, B, gA, gB, kappa, false, far_out + 54 * p);
    if (SYM && lane == 1) expand_blocks(acc, A, B, gA, gB, kappa, true, far_out + 54 * (int64_t)rev[p]);
}

// Coincident pairs (tau, tau). The double layer vanishes (x - y lies in the
// plane of tau), and the single-layer integrand is symmetric in x and y, so
// the three regions of the coincident map whose roles are exchanged (regions
// 3..5) give the transposes of regions 0..2: integrate those and symmetrise.
// Accumulators: S_L[9], S_Y[9], sum w G_L, sum w G_Y. The far rule likewise
// over its point pairs i < j (identical points are skipped by the pair kernel).
__device__ __forceinline__ void accum_v(double* acc, double w, const double* x, const double* y, const double* lx,
                                        const double* ly, double kappa) {
    const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
    const double rinv = rsqrt(r2);
    const double gl = rinv * 0.07957747154594767;  // 1 / (4 pi r)
    const double gy = exp_nonpos(-kappa * (r2 * rinv)) * gl;
    for (int a = 0; a < 3; ++a) {
        const double wa = w * lx[a];
        for (int b = 0; b < 3; ++b) {
            const double ll = wa * ly[b];
            acc[3 * a + b] += gl * ll;
            acc[9 + 3 * a + b] += gy * ll;
        }
    }
    acc[18] += w * gl;
    acc[19] += w * gy;
}

__device__ void expand_coin(const double* acc, const TriFrame& A, const double* tgeoA, double kappa, double* out) {
    const double nn = A.n[0] * A.n[0] + A.n[1] * A.n[1] + A.n[2] * A.n[2];
    const double f = 1.0 / (4.0 * A.area * A.area);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const double* ea = tgeoA + 4 + 3 * a;
            const double* eb = tgeoA + 4 + 3 * b;
            const double cc = f * (ea[0] * eb[0] + ea[1] * eb[1] + ea[2] * eb[2]);
            const int ab = 3 * a + b, ba = 3 * b + a;
            const double vl = acc[ab] + acc[ba], vy = acc[9 + ab] + acc[9 + ba];
            double* e = out + 6 * ab;  // the layout of expand_blocks
            e[0] = vl;
            e[1] = 0.0;
            e[2] = cc * (2.0 * acc[18]);
            e[3] = vy;
            e[4] = 0.0;
            e[5] = cc * (2.0 * acc[19]) + kappa * kappa * nn * vy;
        }
}

__global__ void __launch_bounds__(NEAR_THREADS, 4)
k_coin_pairs(const double* __restrict__ verts, const int32_t* __restrict__ tris, const double* __restrict__ tgeo,
             const int4* __restrict__ pairs, const int32_t* __restrict__ list, int64_t nlist, SSTable tab, int n4,
             Rule rule, double kappa, double* __restrict__ ss_out, double* __restrict__ far_out) {
    __shared__ TriFrame frames[NEAR_THREADS / 32];
    __shared__ double red[NEAR_THREADS / 32][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t li = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (li >= nlist) return;  // whole warps leave together
    const int64_t p = list[li];
    const int4 pr = pairs[p];
    TriFrame& A = frames[wid];
    if (lane == 0) make_frame(verts, tris, tgeo, pr.x, pr.w & 63, A);
    __syncwarp();
    const int e0 = 0;
    const double jac_ab = (2.0 * A.area) * (2.0 * A.area);
    double acc[20];
    {
        double mom[18];
        for (int k = 0; k < 18; ++k) mom[k] = 0.0;
        for (int idx = lane; idx < 3 * n4; idx += 32) accum_coin_frame(mom, tab, e0 + idx, A, kappa);
        warp_allsum<18, 32>(mom, lane, red[wid]);
        for (int k = 0; k < 18; ++k) mom[k] *= jac_ab;
        frame_to_corner(mom, A, A, acc);
        frame_to_corner(mom + 9, A, A, acc + 9);
        acc[18] = mom[0];
        acc[19] = mom[9];
    }
    const double* gA = tgeo + 16 * (int64_t)pr.x;
    if (lane == 0) expand_coin(acc, A, gA, kappa, ss_out + 54 * p);
    for (int k = 0; k < 20; ++k) acc[k] = 0.0;
    const int Q = rule.Q;
    for (int idx = lane; idx < Q * Q; idx += 32) {
        const int i = idx / Q, j = idx % Q;
        if (j <= i) continue;
        double x[3], y[3];
        for (int k = 0; k < 3; ++k) {
            x[k] = rule.l[i][0] * corner(A, 0, k) + rule.l[i][1] * corner(A, 1, k) + rule.l[i][2] * corner(A, 2, k);
            y[k] = rule.l[j][0] * corner(A, 0, k) + rule.l[j][1] * corner(A, 1, k) + rule.l[j][2] * corner(A, 2, k);
        }
        const double w = rule.w[i] * A.area * rule.w[j] * A.area;
        accum_v(acc, w, x, y, rule.l[i], rule.l[j], kappa);
    }
    warp_allsum<20, 32>(acc, lane, red[wid]);
    if (lane == 0) expand_coin(acc, A, gA, kappa, far_out + 54 * p);
}

// Band pairs (share no vertex, closer than the plan's band): the blocks of the
// band rule minus those of the far rule, for the pair and its reverse, one
// thread per band pair (t, s) with t < s. Points are the rules' barycentric
// combinations of the corners, in the corners' original order. Band pair q is
// stored at n_adj + q.
//
// Both rules are products of one triangle rule on each triangle, so every block
// entry factors as sum_i w_i l_a(x_i) [sum_j w_j l_b(y_j) g(x_i, y_j)]: for each
// x point the thread first sums the six kernels against the y points' three
// basis values (18 FMA per point pair), then adds those partial sums into the
// 3x3 blocks (54 FMA per x point). The sums of w G over the pair follow from
// the single-layer blocks, the basis functions summing to one at every point.
// The y points of both rules are staged in shared memory, per thread.
constexpr int BAND_THREADS = 128;

// FP64 flops of one band pair under a Q-point rule by formula count: per point
// pair the kernel evaluation (33, as for the regularised pairs) and the partial
// sums (18 FMA); per point of either triangle its position (15); per x point
// its weights (4) and the block updates (54 FMA).
__host__ __device__ constexpr double band_flops(int Q) { return Q * Q * (33.0 + 36.0) + Q * (30.0 + 4.0 + 108.0); }

template <int Q>
__device__ __forceinline__ void band_pass(double* acc, const double (&pa)[3][3], const double* ys,
                                          const double (*wl)[3], const Rule& R, double wscale, const double* na,
                                          const double* nb, double kappa) {
#pragma unroll 1
    for (int i = 0; i < Q; ++i) {
        double x[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) x[k] = R.l[i][0] * pa[0][k] + R.l[i][1] * pa[1][k] + R.l[i][2] * pa[2][k];
        double u[6][3];
#pragma unroll
        for (int k = 0; k < 6; ++k) u[k][0] = u[k][1] = u[k][2] = 0.0;
#pragma unroll 1
        for (int j = 0; j < Q; ++j) {
            const double d0 = x[0] - ys[(3 * j) * BAND_THREADS], d1 = x[1] - ys[(3 * j + 1) * BAND_THREADS],
                         d2 = x[2] - ys[(3 * j + 2) * BAND_THREADS];
            const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
            const double rinv = rsqrt(r2);
            const double r = r2 * rinv;
            const double gl = rinv * 0.07957747154594767;  // 1 / (4 pi r)
            const double ek = exp_nonpos(-kappa * r);
            const double fl = gl * rinv * rinv;  // 1 / (4 pi r^3)
            const double fy_over_fl = ek * (1.0 + kappa * r);
            const double kl = fl * (d0 * nb[0] + d1 * nb[1] + d2 * nb[2]);
            const double ktl = fl * -(d0 * na[0] + d1 * na[1] + d2 * na[2]);  // (y - x).n_x
            const double g[6] = {gl, ek * gl, kl, kl * fy_over_fl, ktl, ktl * fy_over_fl};
#pragma unroll
            for (int k = 0; k < 6; ++k)
#pragma unroll
                for (int c = 0; c < 3; ++c) u[k][c] += g[k] * wl[j][c];
        }
        // blocks: V_L, V_Y, K_L, K_Y at 0, 9, 18, 27; the reversed pair's K_L, K_Y at 38, 47
        const double wi = wscale * R.w[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double wa = wi * R.l[i][a];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const int base = k < 4 ? 9 * k : 38 + 9 * (k - 4);
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[base + 3 * a + c] += wa * u[k][c];
            }
        }
    }
}

template <int QF, int QC>
__global__ void __launch_bounds__(BAND_THREADS, 2)
k_band_pairs(const double* __restrict__ verts, const int32_t* __restrict__ tris, const double* __restrict__ tgeo,
             const int32_t* __restrict__ band_ptr, const int32_t* __restrict__ band_s,
             const int32_t* __restrict__ band_t, int64_t n_band, int64_t n_adj, Rule fine, Rule coarse, double kappa,
             double* __restrict__ ss_out, int* __restrict__ status) {
    __shared__ double ysm[(QF + QC) * 3 * BAND_THREADS];
    __shared__ double wl[2][6][3];  // w_j l_b(y_j) of the fine and the coarse rule
    if (threadIdx.x < 36) {
        const int r = threadIdx.x / 18, j = (threadIdx.x / 3) % 6, c = threadIdx.x % 3;
        const Rule& R = r == 0 ? fine : coarse;
        wl[r][j][c] = R.w[j] * R.l[j][c];
    }
    __syncthreads();
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n_band) return;  // no barrier follows
    const int32_t pt = band_t[q], ps = band_s[q];
    if (pt > ps) return;  // the reverse of a pair handled by its other thread
    // the reversed pair: t among the partners of s (sorted)
    int32_t lo = band_ptr[ps], hi = band_ptr[ps + 1];
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (band_s[mid] < pt) lo = mid + 1;
        else hi = mid;
    }
    if (lo >= band_ptr[ps + 1] || band_s[lo] != pt) {  // the band lists are symmetric by construction
        atomicExch(status, PB_EMESH);
        return;
    }
    const int64_t p = n_adj + q, pr_rev = n_adj + lo;
    double pa[3][3];
    {
        double pb[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                pa[a][k] = verts[3 * (int64_t)tris[3 * (int64_t)pt + a] + k];
                pb[a][k] = verts[3 * (int64_t)tris[3 * (int64_t)ps + a] + k];
            }
        double* ys = ysm + threadIdx.x;
#pragma unroll
        for (int j = 0; j < QF + QC; ++j) {
            const Rule& R = j < QF ? fine : coarse;
            const int jj = j < QF ? j : j - QF;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                ys[(3 * j + k) * BAND_THREADS] = R.l[jj][0] * pb[0][k] + R.l[jj][1] * pb[1][k] + R.l[jj][2] * pb[2][k];
        }
    }
    const double* gA = tgeo + 16 * (int64_t)pt;
    const double* gB = tgeo + 16 * (int64_t)ps;
    const double na[3] = {gA[0], gA[1], gA[2]}, nb[3] = {gB[0], gB[1], gB[2]};
    double acc[NACC_SYM];
#pragma unroll
    for (int k = 0; k < NACC_SYM; ++k) acc[k] = 0.0;
    const double area2 = gA[3] * gB[3];
    band_pass<QF>(acc, pa, ysm + threadIdx.x, wl[0], fine, area2, na, nb, kappa);
    band_pass<QC>(acc, pa, ysm + threadIdx.x + 3 * QF * BAND_THREADS, wl[1], coarse, -area2, na, nb, kappa);
    double s0 = 0.0, s1 = 0.0;  // sums of w G_L and w G_Y over the pair
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        s0 += acc[k];
        s1 += acc[9 + k];
    }
    acc[36] = s0;
    acc[37] = s1;
    TriFrame A, B;  // expand_blocks reads the normals and areas only
    for (int k = 0; k < 3; ++k) {
        A.n[k] = na[k];
        B.n[k] = nb[k];
    }
    A.area = gA[3];
    B.area = gB[3];
    expand_blocks(acc, A, B, gA, gB, kappa, false, ss_out + 54 * p);
    expand_blocks(acc, A, B, gA, gB, kappa, true, ss_out + 54 * pr_rev);
}

// One warp per row i. The warp walks the contributions of the row in a fixed
// order (the triangles t of i; each one's adjacent pairs, then its band pairs;
// the trial corner b), 32 at a time: each lane finds its contribution's
// column position (binary search in the row's sorted columns) and stages its
// values; then the lane that owns a position (position mod 32) adds the
// staged values for it in slot order. Every entry therefore sums its
// contributions in the walk's order, whatever the scheduling. Adjacent pairs
// (p < n_adj) hold the regularised blocks in ss and the far rule's in far;
// band pairs hold the difference in ss. The row's accumulators (6 operators
// and M) live in shared memory, maxrow entries per warp.
constexpr int ROW_STAGE = 13;  // near[6], full[6] (kept for the diagonal), mass; positions apart (ints)

__device__ __forceinline__ int row_lower_bound(const int32_t* c, int n, int32_t v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (c[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// shared memory of one warp, in doubles
__host__ __device__ inline size_t row_warp_doubles(int maxrow) {
    return 32 * ROW_STAGE + 16 + 7 * (size_t)maxrow + ((size_t)maxrow + 1) / 2;
}

__global__ void k_near_rows(int64_t nv, int64_t nnz, int maxrow, int warps, const int32_t* __restrict__ row_ptr,
                            const int32_t* __restrict__ col, const int32_t* __restrict__ v2t_ptr,
                            const int32_t* __restrict__ v2t, const int32_t* __restrict__ tris,
                            const int32_t* __restrict__ adj_ptr, const int4* __restrict__ pairs,
                            const int32_t* __restrict__ band_ptr, const int32_t* __restrict__ band_s, int64_t n_adj,
                            const double* __restrict__ tgeo, const double* __restrict__ ss,
                            const double* __restrict__ far, double* __restrict__ val, double* __restrict__ diag) {
    extern __shared__ double rsm[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * warps + w;
    if (i >= nv) return;  // whole warps
    double* stage = rsm + (size_t)w * row_warp_doubles(maxrow);
    int32_t* spos = (int32_t*)(stage + 32 * ROW_STAGE);  // 32 ints
    double* acc = stage + 32 * ROW_STAGE + 16;
    int32_t* scol = (int32_t*)(acc + 7 * (size_t)maxrow);
    const int32_t r0 = row_ptr[i];
    const int n = row_ptr[i + 1] - r0;  // <= maxrow
    for (int k = lane; k < n; k += 32) scol[k] = col[r0 + k];
    for (int k = lane; k < 7 * n; k += 32) acc[k] = 0.0;
    __syncwarp();
    const int diag_pos = row_lower_bound(scol, n, (int32_t)i);
    double dfull[6] = {0, 0, 0, 0, 0, 0};  // the diagonal entry's full values (kept by its owner lane)
    for (int32_t k = v2t_ptr[i]; k < v2t_ptr[i + 1]; ++k) {
        const int32_t t = v2t[k] / 3, a = v2t[k] % 3;
        const int32_t p0 = adj_ptr[t], L1 = adj_ptr[t + 1] - p0;
        const int32_t q0 = band_ptr ? band_ptr[t] : 0, L2 = band_ptr ? band_ptr[t + 1] - q0 : 0;
        const int total = 3 * (L1 + L2);
        for (int c0 = 0; c0 < total; c0 += 32) {
            const int c = c0 + lane;
            if (c < total) {
                double* my = stage + lane * ROW_STAGE;
                const int idx = c / 3, b = c - 3 * idx, ab = 3 * a + b;
                if (idx < L1) {
                    const int64_t pp = p0 + idx;
                    const int4 pr = pairs[pp];
                    const int32_t j = tris[3 * (int64_t)pr.y + b];
                    spos[lane] = row_lower_bound(scol, n, j);
                    const double2* s2 = reinterpret_cast<const double2*>(ss + 54 * pp + 6 * ab);
                    const double2* f2 = reinterpret_cast<const double2*>(far + 54 * pp + 6 * ab);
#pragma unroll
                    for (int h = 0; h < 3; ++h) {
                        const double2 sv = s2[h], fv = f2[h];
                        my[2 * h] = sv.x - fv.x;
                        my[2 * h + 1] = sv.y - fv.y;
                        my[6 + 2 * h] = sv.x;
                        my[7 + 2 * h] = sv.y;
                    }
                    my[12] = pr.z == 0 ? tgeo[16 * (int64_t)pr.x + 3] / 12.0 * ((ab % 4 == 0) ? 2.0 : 1.0) : 0.0;
                } else {
                    const int32_t q = q0 + idx - L1;
                    const int64_t pp = n_adj + q;
                    const int32_t j = tris[3 * (int64_t)band_s[q] + b];
                    spos[lane] = row_lower_bound(scol, n, j);
                    const double2* s2 = reinterpret_cast<const double2*>(ss + 54 * pp + 6 * ab);
#pragma unroll
                    for (int h = 0; h < 3; ++h) {
                        const double2 sv = s2[h];
                        my[2 * h] = sv.x;
                        my[2 * h + 1] = sv.y;
                    }
                    for (int o = 0; o < 6; ++o) my[6 + o] = 0.0;  // band pairs never touch the diagonal
                    my[12] = 0.0;
                }
            }
            __syncwarp();
            // the slots this lane owns, then their values in slot order (lanes in parallel)
            const int m = min(32, total - c0);
            unsigned own = 0;
            for (int sl = 0; sl < m; ++sl)
                if ((spos[sl] & 31) == lane) own |= 1u << sl;
            while (own) {
                const int sl = __ffs(own) - 1;
                own &= own - 1;
                const double* st = stage + sl * ROW_STAGE;
                const int pos = spos[sl];
                double* e = acc + 7 * (size_t)pos;
                for (int o = 0; o < 6; ++o) e[o] += st[o];
                e[6] += st[12];
                if (pos == diag_pos)
                    for (int o = 0; o < 6; ++o) dfull[o] += st[6 + o];
            }
            __syncwarp();
        }
    }
    const int map[6] = {N_VL, N_KL, N_DL, N_VY, N_KY, N_DY};
    for (int k = lane; k < n; k += 32) {
        const double* e = acc + 7 * (size_t)k;
        for (int o = 0; o < 6; ++o) val[map[o] * nnz + r0 + k] = e[o];
        val[N_M * nnz + r0 + k] = e[6];
        if (k == diag_pos) {
            for (int o = 0; o < 6; ++o) diag[map[o] * nv + i] = dfull[o];
            diag[N_M * nv + i] = e[6];
        }
    }
}

// The mass matrix on its own pattern: the entries of each row whose mass value
// is not zero (exactly the vertices sharing a triangle with the row's).
__global__ void k_mass_rows(int64_t nv, int64_t nnz, int pass, const int32_t* __restrict__ row_ptr,
                            const int32_t* __restrict__ col, const double* __restrict__ val,
                            int32_t* __restrict__ cnt, const int32_t* __restrict__ mrow_ptr,
                            int32_t* __restrict__ mcol, double* __restrict__ mval) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nv) return;
    const double* mv = val + N_M * nnz;
    int n = 0;
    for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
        if (mv[k] == 0.0) continue;
        if (pass) {
            mcol[mrow_ptr[i] + n] = col[k];
            mval[mrow_ptr[i] + n] = mv[k];
        }
        ++n;
    }
    if (!pass) cnt[i] = n;
}

static void free_near(pb_near* nf) {
    if (nf->val) cudaFree(nf->val);
    if (nf->diag) cudaFree(nf->diag);
    if (nf->mrow_ptr) cudaFree(nf->mrow_ptr);
    nf->val = nf->diag = nullptr;
    nf->mrow_ptr = nullptr;
}

static int build(pb_ctx* ctx, const pb_mesh* m, double kappa, pb_near* nf, cudaStream_t s) {
    nf->mesh = m;
    nf->kappa = kappa;
    PB_TRY(dev_alloc((void**)&nf->val, sizeof(double) * N_VALS * m->nnz));
    PB_TRY(dev_alloc((void**)&nf->diag, sizeof(double) * N_VALS * m->nv));
    double *ss = nullptr, *far = nullptr;
    int rc = dev_alloc((void**)&ss, sizeof(double) * 54 * m->npairs);
    if (rc == PB_OK) rc = dev_alloc((void**)&far, sizeof(double) * 54 * m->n_adj);
    if (rc == PB_OK) {
        // coincident pairs: the table of their regularised rule
        const int nc = m->n_ss_cls[0], ne = m->n_ss_cls[1], nvx = m->n_ss_cls[2];
        const Gauss gq = gauss01(nc);
        const int n4i = nc * nc * nc * nc, ntab = 3 * n4i;
        // edge and vertex pairs: the outer entries of their maps, each with its own rule
        const int nout_e = 6 * ne * ne * ne, nout_v = 2 * nvx * nvx * nvx;
        const size_t bt = sizeof(double) * SS_TABLE_ARRAYS * ntab;
        const size_t be = sizeof(double) * ((size_t)SS_OUTER_ARRAYS * nout_e + 2 * ne);
        const size_t bv = sizeof(double) * ((size_t)SS_OUTER_ARRAYS * nout_v + 2 * nvx);
        double* tabm = nullptr;
        rc = dev_alloc((void**)&tabm, bt + be + bv);
        if (rc != PB_OK) {
            cudaFree(ss);
            cudaFree(far);
            return rc;
        }
        double* tabe = tabm + bt / sizeof(double);
        double* tabv = tabe + be / sizeof(double);
        k_ss_table<<<(ntab + 127) / 128, 128, 0, s>>>(gq, ntab, tabm);
        k_ss_outer<<<(std::max(nout_e, 2 * ne) + 127) / 128, 128, 0, s>>>(gauss01(ne), 1, nout_e, tabe);
        k_ss_outer<<<(std::max(nout_v, 2 * nvx) + 127) / 128, 128, 0, s>>>(gauss01(nvx), 2, nout_v, tabv);
        ::pb::count_launch(3);
        SSTable tab = {tabm, tabm + ntab, tabm + 2 * ntab, tabm + 3 * ntab, tabm + 4 * ntab, tabm + 5 * ntab, ntab};
        const SSOuter outer_e = {tabe, nout_e, ne, 6}, outer_v = {tabv, nout_v, nvx, 2};
        int threads = NEAR_THREADS;  // one warp per pair
        // coincident pairs, then one of each pair of reversed pairs (which also writes the other)
        unsigned bc = (unsigned)((m->n_coin * 32 + threads - 1) / threads);
        // quadrature point pairs of each kernel, for the profile (formula flop counts per pair in
        // NEAR_FLOPS_*: kernel evaluation and accumulation, a fused multiply-add counted as two)
        const double n4 = (double)n4i, Q = m->Q, Qb = m->Qr;
        if (bc) {
            Timer tm(ctx, PB_KERNEL_NEAR_COIN, s, m->n_coin * (3.0 * n4 + Q * (Q - 1) / 2), NEAR_FLOPS_COIN);
            k_coin_pairs<<<bc, threads, 0, s>>>(m->verts, m->tris, m->tgeo, m->pairs, m->pair_coin, m->n_coin, tab,
                                                n4i, mesh_rule(m), kappa, ss, far);
            tm.stop();
        }
        ::pb::count_launch();
        // edge-adjacent pairs (the first n_prim_edge of the primary list), then vertex-adjacent ones
        for (int cls = 0; cls < 2; ++cls) {
            const int64_t nlist = cls == 0 ? m->n_prim_edge : m->n_prim - m->n_prim_edge;
            if (nlist == 0) continue;
            const int32_t* list = m->pair_prim + (cls == 0 ? 0 : m->n_prim_edge);
            const SSOuter& ot = cls == 0 ? outer_e : outer_v;
            const unsigned bp = (unsigned)((nlist * 32 + threads - 1) / threads);
            const double outer_pts = (double)nlist * ot.n;
            const double reg = outer_pts * ot.nss, farp = (double)nlist * Q * Q;
            const double flops = reg * NEAR_FLOPS_ADJ_POINT + outer_pts * NEAR_FLOPS_ADJ_OUTER + farp * NEAR_FLOPS_SYM;
            Timer tm(ctx, PB_KERNEL_NEAR_ADJ, s, reg + farp, flops / (reg + farp));
#define PB_NEAR_ARGS m->verts, m->tris, m->tgeo, m->pairs, list, nlist, m->pair_rev, ot, mesh_rule(m), kappa, ss, far
            if (ot.nss == 4) k_near_pairs<2, true, 4><<<bp, threads, 0, s>>>(PB_NEAR_ARGS);
            else if (ot.nss == 3) k_near_pairs<2, true, 3><<<bp, threads, 0, s>>>(PB_NEAR_ARGS);
            else k_near_pairs<2, true, 0><<<bp, threads, 0, s>>>(PB_NEAR_ARGS);
#undef PB_NEAR_ARGS
            ::pb::count_launch();
            tm.stop();
        }
        if (m->n_band) {
            Rule fine = mesh_ref_rule(m), coarse = mesh_rule(m);
            const double ppairs = 0.5 * m->n_band * (Qb * Qb + Q * Q);
            Timer tm(ctx, PB_KERNEL_NEAR_BAND, s, ppairs,
                     0.5 * m->n_band * (band_flops(m->Qr) + band_flops(m->Q)) / ppairs);
            const unsigned gb = (unsigned)((m->n_band + BAND_THREADS - 1) / BAND_THREADS);
#define PB_BAND_ARGS m->verts, m->tris, m->tgeo, m->band_ptr, m->band_s, m->band_t, m->n_band, m->n_adj, fine, \
                     coarse, kappa, ss, m->status
            if (m->Qr == 6 && m->Q == 3) k_band_pairs<6, 3><<<gb, BAND_THREADS, 0, s>>>(PB_BAND_ARGS);
            else if (m->Qr == 6 && m->Q == 1) k_band_pairs<6, 1><<<gb, BAND_THREADS, 0, s>>>(PB_BAND_ARGS);
            else if (m->Qr == 3 && m->Q == 1) k_band_pairs<3, 1><<<gb, BAND_THREADS, 0, s>>>(PB_BAND_ARGS);
            else rc = set_error(PB_EINVAL, "band rule %d with far rule %d", m->Qr, m->Q);
#undef PB_BAND_ARGS
            tm.stop();
            ::pb::count_launch();
        }
        cudaMemsetAsync(nf->diag, 0, sizeof(double) * N_VALS * m->nv, s);
        {
            const size_t per_warp = sizeof(double) * row_warp_doubles(m->max_row);
            const int warps = (int)std::max<size_t>(1, std::min<size_t>(8, (200u << 10) / per_warp));
            const size_t sm = per_warp * warps;
            if (sm > (227u << 10)) {
                rc = set_error(PB_EINVAL, "near pattern rows too long (%d entries) for one warp's shared memory",
                               m->max_row);
            } else {
                // the largest allowed (227 KB), not this launch's sm: builds on other host threads
                // set the same value, so none lowers it under another's launch
                cudaFuncSetAttribute(k_near_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 << 10);
                k_near_rows<<<(unsigned)((m->nv + warps - 1) / warps), 32 * warps, sm, s>>>(
                    m->nv, m->nnz, m->max_row, warps, m->row_ptr, m->col, m->v2t_ptr, m->v2t, m->tris, m->adj_ptr,
                    m->pairs, m->n_band ? m->band_ptr : nullptr, m->band_s, m->n_adj, m->tgeo, ss, far, nf->val,
                    nf->diag);
                ::pb::count_launch();
            }
        }
        // the mass matrix on its own pattern (one allocation: pointers, columns, values)
        if (rc == PB_OK) {
            const int64_t nv = m->nv, cap = m->nnz;
            const size_t bytes = sizeof(int32_t) * (2 * (nv + 1) + cap) + sizeof(double) * (cap + 2) + 64;
            rc = dev_alloc((void**)&nf->mrow_ptr, bytes);
            if (rc == PB_OK) {
                int32_t* cnt = nf->mrow_ptr + (nv + 1);
                nf->mcol = cnt + (nv + 1);
                int64_t* total = (int64_t*)(((uintptr_t)(nf->mcol + cap) + 15) & ~(uintptr_t)15);
                nf->mval = (double*)(total + 1);
                const unsigned nb = (unsigned)((nv + 127) / 128);
                k_mass_rows<<<nb, 128, 0, s>>>(nv, m->nnz, 0, m->row_ptr, m->col, nf->val, cnt, nullptr, nullptr,
                                               nullptr);
                ::pb::count_launch();
                rc = device_scan(nv, cnt, nf->mrow_ptr, total, s);
                k_mass_rows<<<nb, 128, 0, s>>>(nv, m->nnz, 1, m->row_ptr, m->col, nf->val, nullptr, nf->mrow_ptr,
                                               nf->mcol, nf->mval);
                ::pb::count_launch();
            }
        }
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        int st = 0;
        if (e == cudaSuccess && m->n_band) e = cudaMemcpy(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = set_error(PB_ECUDA, "near build: %s", cudaGetErrorString(e));
        else if (st == PB_EMESH) rc = set_error(PB_EMESH, "internal: band pair without reverse");
        cudaFree(tabm);
    }
    if (ss) cudaFree(ss);
    if (far) cudaFree(far);
    return rc;
}

}  // namespace pb

using namespace pb;

extern "C" int pb_near_build(pb_ctx* ctx, const pb_mesh* mesh, double kappa, pb_near** out, void* stream) {
    if (!ctx || !mesh || !out) return set_error(PB_EINVAL, "pb_near_build: NULL argument");
    if (!(kappa >= 0.0) || !std::isfinite(kappa)) return set_error(PB_EINVAL, "kappa must be >= 0");
    *out = nullptr;
    PB_CUDA(cudaSetDevice(ctx->device));
    pb_near* nf = new pb_near();
    int rc = build(ctx, mesh, kappa, nf, (cudaStream_t)stream);
    if (rc != PB_OK) {
        free_near(nf);
        delete nf;
        return rc;
    }
    *out = nf;
    return PB_OK;
}

namespace pb {
__global__ void k_exp_selftest(const double* __restrict__ x, double* __restrict__ y, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = exp_nonpos(x[i]);
}
}  // namespace pb

extern "C" int pb_selftest_exp(pb_ctx* ctx, const double* x, double* y, int64_t n, void* stream) {
    if (!ctx || (n > 0 && (!x || !y)) || n < 0) return set_error(PB_EINVAL, "pb_selftest_exp: bad argument");
    if (n == 0) return PB_OK;
    PB_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    k_exp_selftest<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, y, n);
    ::pb::count_launch();
    PB_CUDA(cudaGetLastError());
    PB_CUDA(cudaStreamSynchronize(s));
    return PB_OK;
}

extern "C" int pb_free_near(pb_near* nf) {
    if (!nf) return PB_OK;
    free_near(nf);
    delete nf;
    return PB_OK;
}
