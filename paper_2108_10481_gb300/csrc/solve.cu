// a7 + a8 + a9: preconditioners, GMRES and mixed-precision refinement, and the
// public operator-application calls.
//
// Paper, "Preconditioning": left preconditioning P^-1 A x = P^-1 b solved by
// GMRES; block-diagonal (algebraic), mass and scaled-mass (eqs. prec:mass,
// prec:mass:scaled) and Calderon (eqs. prec:calderon:int, prec:calderon:ext)
// preconditioners. Products of weak-form operators carry M^-1 in between
// (strong form), and the outer mass matrix is inverted on the left.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "solver.h"

namespace pb {

int rhs_coefs(const pb_params* prm, int form, double alpha, double beta, double d[2], double n[2]);
int half_calderon_scaling(const pb_params* prm, int form, int which, double* a, double* b);

// ----------------------------------------------------------- vector kernels
__global__ void k_copy(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = x[i];
}
__global__ void k_scale_halves(int64_t nv, double a, double b, double* __restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < 2 * nv) y[i] *= (i < nv) ? a : b;
}
__global__ void k_sub(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                      double* __restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = a[i] - b[i];
}
__global__ void k_add_inplace(int64_t n, const double* __restrict__ a, double* __restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] += a[i];
}

// block diagonal: per-DOF inverse of [[A00_ii, A01_ii], [A10_ii, A11_ii]]
__global__ void k_block_diag_setup(int64_t nv, const double* __restrict__ diag, BlockOp B,
                                   double* __restrict__ inv) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nv) return;
    double dv[O_N];
    dv[O_M] = diag[N_M * nv + i];
    dv[O_VL] = diag[N_VL * nv + i];
    dv[O_KL] = diag[N_KL * nv + i];
    dv[O_TL] = dv[O_KL];  // the diagonal of K^T is the diagonal of K
    dv[O_DL] = diag[N_DL * nv + i];
    dv[O_VY] = diag[N_VY * nv + i];
    dv[O_KY] = diag[N_KY * nv + i];
    dv[O_TY] = dv[O_KY];
    dv[O_DY] = diag[N_DY * nv + i];
    double a[2][2];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double s = 0.0;
            for (int o = 0; o < O_N; ++o) s += B.c[r][c][o] * dv[o];
            a[r][c] = s;
        }
    double det = a[0][0] * a[1][1] - a[0][1] * a[1][0];
    inv[4 * i + 0] = a[1][1] / det;
    inv[4 * i + 1] = -a[0][1] / det;
    inv[4 * i + 2] = -a[1][0] / det;
    inv[4 * i + 3] = a[0][0] / det;
}
__global__ void k_block_diag_apply(int64_t nv, const double* __restrict__ inv, const double* __restrict__ x,
                                   double* __restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nv) return;
    double u = x[i], v = x[nv + i];
    y[i] = inv[4 * i] * u + inv[4 * i + 1] * v;
    y[nv + i] = inv[4 * i + 2] * u + inv[4 * i + 3] * v;
}

// ------------------------------------------------- mass solve (Chebyshev)
// The Jacobi-preconditioned P1 mass matrix has its spectrum in [1/2, 2]: the
// element matrix |tau|/12 [[2,1,1],[1,2,1],[1,1,2]] against its diagonal has
// eigenvalues {2, 1/2, 1/2}, and assembly keeps the Rayleigh quotient in that
// interval. Chebyshev iteration on that interval needs no inner products.
constexpr double CH_LO = 0.5, CH_HI = 2.0;

__global__ void k_cheb_init(int64_t nv, const double* __restrict__ mdiag, const double* __restrict__ b,
                            double* __restrict__ x, double* __restrict__ r, double* __restrict__ d, double theta) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 2 * nv) return;
    int64_t row = i < nv ? i : i - nv;
    r[i] = b[i];
    x[i] = 0.0;
    d[i] = b[i] / (theta * mdiag[row]);
}
// one thread per vertex: row i of both halves (they share the pattern and values)
__global__ void k_cheb_step(int64_t nv, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const double* __restrict__ mval, const double* __restrict__ mdiag,
                            const double* __restrict__ d, double* __restrict__ dn, double* __restrict__ x,
                            double* __restrict__ r, double c_d, double c_r) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nv) return;
    double md0 = 0.0, md1 = 0.0;
    for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
        const double mv = mval[k];
        const int32_t c = col[k];
        md0 += mv * d[c];
        md1 += mv * d[nv + c];
    }
    const double md[2] = {md0, md1};
    const double inv = mdiag[i];
    for (int h = 0; h < 2; ++h) {
        const int64_t ii = i + h * nv;
        const double rn = r[ii] - md[h];
        x[ii] += d[ii];
        r[ii] = rn;
        dn[ii] = c_d * d[ii] + c_r * rn / inv;
    }
}

int mass_solve(const pb_mesh* m, const pb_near* nf, const double* b, double* x, double* work, int iters,
               cudaStream_t s) {
    const int64_t nv = m->nv, n2 = 2 * nv;
    double* r = work;
    double* d0 = work + n2;
    double* d1 = work + 2 * n2;
    const double theta = 0.5 * (CH_HI + CH_LO), delta = 0.5 * (CH_HI - CH_LO), sigma = theta / delta;
    const double* mval = nf->mval;  // the mass matrix on its own pattern
    const double* mdiag = nf->diag + N_M * nv;
    unsigned blocks = (unsigned)((n2 + 255) / 256);
    k_cheb_init<<<blocks, 256, 0, s>>>(nv, mdiag, b, x, r, d0, theta); ::pb::count_launch();
    // algorithmic bytes of one step: the mass pattern once (row pointers, columns and
    // values; nv + 3 nt entries on a closed surface) and its diagonal, d read, the
    // next d written, x and r read and written (2 nv doubles each)
    const double mnnz = (double)nv + 3.0 * (double)m->nt;
    const double step_bytes = 4.0 * (double)(nv + 1) + 12.0 * mnnz + 8.0 * (double)nv + 6.0 * 8.0 * (double)n2;
    double rho = 1.0 / sigma;
    for (int k = 0; k < iters; ++k) {
        double rho_n = 1.0 / (2.0 * sigma - rho);
        Timer tm(m->ctx, PB_KERNEL_CHEB, s, step_bytes, 1.0);
        k_cheb_step<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(nv, nf->mrow_ptr, nf->mcol, mval, mdiag, d0, d1, x,
                                                                  r, rho_n * rho, 2.0 * rho_n / delta);
        ::pb::count_launch();
        tm.stop();
        rho = rho_n;
        double* t = d0;
        d0 = d1;
        d1 = t;
    }
    k_add_inplace<<<blocks, 256, 0, s>>>(n2, d0, x); ::pb::count_launch();
    PB_CUDA(cudaGetLastError());
    return PB_OK;
}

// --------------------------------------------------------------- GMRES kernels
constexpr int DOT_THREADS = 256;
constexpr int DOT_CHUNK = 2048;

// part[k * nchunk + c] = sum over chunk c of V[k] . w
__global__ void k_dots(int64_t n, const double* __restrict__ V, int64_t ldv, const double* __restrict__ w,
                       double* __restrict__ part, int nchunk) {
    __shared__ double red[DOT_THREADS / 32];
    int k = blockIdx.y;
    int c = blockIdx.x;
    const double* vk = V + (int64_t)k * ldv;
    int64_t i0 = (int64_t)c * DOT_CHUNK;
    int64_t i1 = min(n, i0 + DOT_CHUNK);
    double s = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += DOT_THREADS) s += vk[i] * w[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int j = 0; j < DOT_THREADS / 32; ++j) t += red[j];
        part[(int64_t)k * nchunk + c] = t;
    }
}
// out[k] = sum_c part[k * nchunk + c] (fixed order); optionally accumulate
__global__ void k_dots_finish(int nk, int nchunk, const double* __restrict__ part, double* __restrict__ out,
                              int accumulate) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nk) return;
    double t = 0.0;
    for (int c = 0; c < nchunk; ++c) t += part[(int64_t)k * nchunk + c];
    out[k] = accumulate ? out[k] + t : t;
}
// w -= sum_k V[k] h[k]  (sign = -1) or x += sum_k V[k] h[k] (sign = +1)
__global__ void k_vh(int64_t n, int nk, const double* __restrict__ V, int64_t ldv, const double* __restrict__ h,
                     double sign, double* __restrict__ w) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int k = 0; k < nk; ++k) s += V[(int64_t)k * ldv + i] * h[k];
    w[i] += sign * s;
}
// ---- one Arnoldi step with the iteration index j read from the device
constexpr int DOT_KY = 32;  // grid rows of the Gram-Schmidt dots (stride over k <= j)

// part[k * nchunk + c] = chunk c of V[k] . w for k = 0..j
__global__ void k_dots_j(int64_t n, const double* __restrict__ V, const double* __restrict__ w,
                         double* __restrict__ part, int nchunk, const int* __restrict__ jdev) {
    __shared__ double red[DOT_THREADS / 32];
    const int j = *jdev;
    const int c = blockIdx.x;
    const int64_t i0 = (int64_t)c * DOT_CHUNK;
    const int64_t i1 = min(n, i0 + DOT_CHUNK);
    for (int k = blockIdx.y; k <= j; k += gridDim.y) {
        const double* vk = V + (int64_t)k * n;
        double s = 0.0;
        for (int64_t i = i0 + threadIdx.x; i < i1; i += DOT_THREADS) s += vk[i] * w[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < DOT_THREADS / 32; ++q) t += red[q];
            part[(int64_t)k * nchunk + c] = t;
        }
        __syncthreads();
    }
}
// pass 0: column j of H; pass 1: y (the second Gram-Schmidt pass); k = 0..j
__global__ void k_dots_finish_j(int nchunk, const double* __restrict__ part, double* __restrict__ H, int ldh,
                                double* __restrict__ y, const int* __restrict__ jdev, int pass) {
    const int j = *jdev;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > j) return;
    double t = 0.0;
    for (int c = 0; c < nchunk; ++c) t += part[(int64_t)k * nchunk + c];
    if (pass == 0) H[(int64_t)j * ldh + k] = t;
    else y[k] = t;
}
// w -= sum_{k<=j} V[k] c[k], c = column j of H (pass 0) or y (pass 1)
__global__ void k_vh_j(int64_t n, const double* __restrict__ V, const double* __restrict__ H, int ldh,
                       const double* __restrict__ y, const int* __restrict__ jdev, int pass, double* __restrict__ w) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = *jdev;
    const double* c = pass == 0 ? H + (int64_t)j * ldh : y;
    double s = 0.0;
    for (int k = 0; k <= j; ++k) s += V[(int64_t)k * n + i] * c[k];
    w[i] -= s;
}
// column j of H += y (the second pass's coefficients); H[j+1, j] = ||w||^2
__global__ void k_hcol_j(int nchunk, const double* __restrict__ part, double* __restrict__ H, int ldh,
                         const double* __restrict__ y, const int* __restrict__ jdev) {
    const int j = *jdev;
    double* h = H + (int64_t)j * ldh;
    for (int k = threadIdx.x; k <= j; k += blockDim.x) h[k] += y[k];
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int c = 0; c < nchunk; ++c) t += part[c];
        h[j + 1] = t;
    }
}
// V[j+1] = vin = w / ||w|| (zero vector on breakdown)
__global__ void k_normalize_j(int64_t n, const double* __restrict__ w, const double* __restrict__ H, int ldh,
                              const int* __restrict__ jdev, double* __restrict__ V, double* __restrict__ vin) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = *jdev;
    const double nrm = sqrt(H[(int64_t)j * ldh + j + 1]);
    const double v = nrm > 1e-300 ? w[i] / nrm : 0.0;
    V[(int64_t)(j + 1) * n + i] = v;
    vin[i] = v;
}
// Givens rotations on column j of H (column-major, ldh = m + 1) and on g;
// res[0] = |g[j+1]| / beta, res[1] = the new diagonal; then j += 1
__global__ void k_givens_j(double* __restrict__ H, int ldh, double* __restrict__ cs, double* __restrict__ sn,
                           double* __restrict__ g, const double* __restrict__ beta, double* __restrict__ res,
                           int* __restrict__ jdev) {
    const int j = *jdev;
    double* h = H + (int64_t)j * ldh;
    h[j + 1] = sqrt(h[j + 1]);
    for (int i = 0; i < j; ++i) {
        double t = cs[i] * h[i] + sn[i] * h[i + 1];
        h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = t;
    }
    double a = h[j], b = h[j + 1];
    double den = hypot(a, b);
    double c = den > 0.0 ? a / den : 1.0, s = den > 0.0 ? b / den : 0.0;
    cs[j] = c;
    sn[j] = s;
    h[j] = den;
    h[j + 1] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    res[0] = fabs(g[j + 1]) / beta[0];
    res[1] = den;
    *jdev = j + 1;
}
// g = beta e1, beta = sqrt(n2[0]), j = 0
__global__ void k_gm_begin(const double* __restrict__ n2, double* __restrict__ g, double* __restrict__ beta,
                           int* __restrict__ jdev) {
    const double b = sqrt(n2[0]);
    g[0] = b;
    beta[0] = b;
    *jdev = 0;
}
// V[0] = vin = w / beta
__global__ void k_normalize0(int64_t n, const double* __restrict__ w, const double* __restrict__ n2,
                             double* __restrict__ V, double* __restrict__ vin) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double nrm = sqrt(n2[0]);
    const double v = nrm > 1e-300 ? w[i] / nrm : 0.0;
    V[i] = v;
    vin[i] = v;
}

// back substitution R y = g (R upper triangular k x k in H)
__global__ void k_backsolve(int k, const double* __restrict__ H, int ldh, const double* __restrict__ g,
                            double* __restrict__ y) {
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int c = i + 1; c < k; ++c) s -= H[(int64_t)c * ldh + i] * y[c];
        double d = H[(int64_t)i * ldh + i];
        y[i] = d != 0.0 ? s / d : 0.0;
    }
}

// ------------------------------------------------------------------- solver
static unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

// Chebyshev steps of the mass solves inside FP32 (inner) applications: the
// error after k steps is below 2 ((sqrt(kappa) - 1) / (sqrt(kappa) + 1))^k with
// kappa = 4 for the Jacobi-scaled P1 mass matrix, i.e. 2 / 3^k: 4.6e-8 at 16,
// under the FP32 operator's own rounding. FP64 and accurate applications (the
// outer residual's norm) keep the full count.
constexpr int CHEB_ITERS_F32 = 16;

static int cheb_count(const Solver& S, int prec) {
    return prec == PB_F32 ? std::min(S.cheb_iters, CHEB_ITERS_F32) : S.cheb_iters;
}

// y = P^-1 x
int apply_prec(Solver& S, int prec, const double* x, double* y) {
    const pb_mesh* m = S.m;
    const int64_t nv = m->nv, n2 = 2 * nv;
    const int ci = cheb_count(S, prec);
    switch (S.pc) {
        case PB_PC_NONE:
            k_copy<<<nb(n2), 256, 0, S.s>>>(n2, x, y); ::pb::count_launch();
            break;
        case PB_PC_BLOCK_DIAG:
            k_block_diag_apply<<<nb(nv), 256, 0, S.s>>>(nv, S.bdiag, x, y); ::pb::count_launch();
            break;
        case PB_PC_MASS:
        case PB_PC_SCALED_MASS:
            PB_TRY(mass_solve(m, S.nf, x, y, S.cheb, ci, S.s));
            break;
        default:  // Calderon: M^-1 C M^-1
            PB_TRY(mass_solve(m, S.nf, x, S.t1, S.cheb, ci, S.s));
            {
                const double* cc = nullptr;
                PB_TRY(solver_comb(S, true, &cc));
                PB_TRY(apply_blockop(S.mc, S.nc, S.C, prec, S.t1, S.t2, S.s, cc));
            }
            S.applies++;
            PB_TRY(mass_solve(m, S.nf, S.t2, y, S.cheb, ci, S.s));
            break;
    }
    if (S.sa != 1.0 || S.sb != 1.0) {
        k_scale_halves<<<nb(n2), 256, 0, S.s>>>(nv, 1.0 / S.sa, 1.0 / S.sb, y);
        ::pb::count_launch();
    }
    PB_CUDA(cudaGetLastError());
    return PB_OK;
}

// y = P^-1 A x
static int apply_op(Solver& S, int prec, const double* x, double* y) {
    const double* ca = nullptr;
    PB_TRY(solver_comb(S, false, &ca));
    PB_TRY(apply_blockop(S.m, S.nf, S.A, prec, x, S.t3, S.s, ca));
    S.applies++;
    return apply_prec(S, prec, S.t3, y);
}

int gmres_alloc(GmresWork& G, int64_t n, int mmax) {
    const size_t nchunk = (size_t)((n + DOT_CHUNK - 1) / DOT_CHUNK);
    const size_t m = (size_t)mmax;
    // offsets (in doubles) of every array, then one allocation of the total
    const size_t oV = 0, ow = oV + (m + 1) * n, oH = ow + n, ocs = oH + (m + 1) * m, osn = ocs + m,
                 oy = osn + m, og = oy + m, opart = og + m + 2, ores = opart + (m + 2) * nchunk,
                 ovin = ores + 16, ojd = ovin + n, total = ojd + 2;
    PB_TRY(dev_alloc(&G.block, sizeof(double) * total));
    double* p = (double*)G.block;
    G.V = p + oV;
    G.w = p + ow;
    G.H = p + oH;
    G.cs = p + ocs;
    G.sn = p + osn;
    G.y = p + oy;
    G.g = p + og;
    G.part = p + opart;
    G.res = p + ores;  // res[0..1] estimates, res[2..3] scratch, res[4] beta
    G.vin = p + ovin;
    G.jdev = (int*)(p + ojd);
    G.mmax = mmax;
    G.n = n;
    return PB_OK;
}
void gmres_free(GmresWork& G) {
    if (G.block) cudaFree(G.block);
    G.block = nullptr;
}

// out[0..nk) = V[0..nk) . w   (accumulate: out += ...)
void dots(GmresWork& G, const double* V, int nk, const double* w, double* out, int accumulate, cudaStream_t s) {
    int nchunk = (int)((G.n + DOT_CHUNK - 1) / DOT_CHUNK);
    dim3 grid(nchunk, nk);
    k_dots<<<grid, DOT_THREADS, 0, s>>>(G.n, V, G.n, w, G.part, nchunk); ::pb::count_launch();
    k_dots_finish<<<(nk + 127) / 128, 128, 0, s>>>(nk, nchunk, G.part, out, accumulate); ::pb::count_launch();
}

// One GMRES iteration: w = P^-1 A V[j], then the Arnoldi step.
static int gm_iteration(Solver& S, GmresWork& G, int prec) {
    PB_TRY(apply_op(S, prec, G.vin, G.w));
    return gm_step(G, G.w, G.res, S.s);
}

// The iteration from its CUDA graph: captured at the second iteration (the
// first has reserved every workspace) and replayed from then on.
static int iterate(Solver& S, GmresWork& G, int prec, int j, StepGraph** replayed) {
    *replayed = nullptr;
    StepGraph& g = S.step[prec & 3];
    const uint64_t* d0 = &S.m->ws_gen;
    const uint64_t* d1 = S.mc != S.m ? &S.mc->ws_gen : nullptr;
    graph_check(g, d0, d1);
    if (!S.graphs || g.failed || (j == 0 && !g.exec)) return gm_iteration(S, G, prec);
    if (!g.exec) {
        const int a0 = S.applies;
        PhaseTrace tr("gmres");
        PB_TRY(graph_capture(g, S.s, [&] { return gm_iteration(S, G, prec); }, d0, d1));
        tr.lap("capture");
        g.applies = S.applies - a0;
        S.applies = a0;
        if (g.failed) return gm_iteration(S, G, prec);
    }
    PB_TRY(graph_replay(g, S.s));
    S.applies += g.applies;
    *replayed = &g;
    return PB_OK;
}

void solver_release(Solver& S) {
    for (auto& g : S.step) graph_free(g);
    if (S.combA) cudaFree(S.combA);
    if (S.combC) cudaFree(S.combC);
    S.combA = S.combC = nullptr;
}

// The near values combined for a block operator depend only on the near field
// and the operator's coefficients, both fixed for a solve: combined once, on the
// first application (before any iteration is captured into a graph), instead of
// once per application.
int solver_comb(Solver& S, bool calderon, const double** out) {
    double*& c = calderon ? S.combC : S.combA;
    if (!c) {
        const pb_mesh* m = calderon ? S.mc : S.m;
        const pb_near* nf = calderon ? S.nc : S.nf;
        const BlockOp& B = calderon ? S.C : S.A;
        PB_TRY(dev_alloc((void**)&c, (sizeof(double) + sizeof(float)) * 4 * (size_t)m->nnz));
        PB_TRY(combine_near(m, nf, B, c, (float*)(c + 4 * m->nnz), S.s));
    }
    *out = c;
    return PB_OK;
}

// Left-preconditioned GMRES on A x = b from x (in/out; x_zero says x = 0, so
// the first residual needs no operator application). Convergence is measured
// as ||P^-1 (b - A x)|| / ref with ref = the initial residual norm when
// ref <= 0. Returns the iterations, the final estimate and the initial norm.
static int gmres(Solver& S, GmresWork& G, int prec, const double* b, double* x, bool x_zero, double tol,
                 double ref, int max_it, int* iters, double* res_out, double* beta_out) {
    const int64_t n = G.n;
    cudaStream_t s = S.s;
    *iters = 0;
    if (x_zero) {
        PB_TRY(apply_prec(S, prec, b, G.w));
    } else {
        const double* ca = nullptr;
        PB_TRY(solver_comb(S, false, &ca));
        PB_TRY(apply_blockop(S.m, S.nf, S.A, prec, x, S.t3, s, ca));
        S.applies++;
        k_sub<<<nb(n), 256, 0, s>>>(n, b, S.t3, S.t2); ::pb::count_launch();
        PB_TRY(apply_prec(S, prec, S.t2, G.w));
    }
    double* scratch = G.res + 2;  // scratch[1] = ||w||^2
    dots(G, G.w, 1, G.w, scratch + 1, 0, s);
    double beta2 = 0.0;
    PB_CUDA(cudaMemcpyAsync(&beta2, scratch + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    PB_CUDA(cudaStreamSynchronize(s));
    const double beta = sqrt(beta2);
    if (beta_out) *beta_out = beta;
    const double denom = ref > 0.0 ? ref : beta;
    *res_out = denom > 0.0 ? beta / denom : 0.0;
    if (!std::isfinite(beta)) return set_error(PB_ENUMERIC, "GMRES: initial residual is not finite");
    if (beta == 0.0 || *res_out <= tol || max_it <= 0) return PB_OK;
    PB_TRY(gm_begin(G, G.w, scratch + 1, s));
    int k = 0;
    double res = *res_out;
    const int mmax = std::min(max_it, G.mmax);
    for (int j = 0; j < mmax; ++j) {
        StepGraph* g = nullptr;
        arnoldi_j() = j;
        PB_TRY(iterate(S, G, prec, j, &g));
        double hr[2];
        PB_CUDA(cudaMemcpyAsync(hr, G.res, sizeof(hr), cudaMemcpyDeviceToHost, s));
        PB_CUDA(cudaStreamSynchronize(s));
        if (g && S.m->ctx->profile) PB_TRY(graph_credit(S.m->ctx, *g, j));
        k = j + 1;
        res = hr[0] * beta / denom;
        if (!std::isfinite(res)) {
            *iters = k;
            *res_out = res;
            return set_error(PB_ENUMERIC, "GMRES: residual is not finite at iteration %d", k);
        }
        if (res <= tol || hr[1] == 0.0) break;
    }
    PB_TRY(gm_finish(G, k, x, s));
    *iters = k;
    *res_out = res;
    return PB_OK;
}

int setup_solver(Solver& S, const pb_mesh* m, const pb_near* nf, const pb_params* prm, int form, int pc,
                        const pb_solve_opts* o, cudaStream_t s) {
    S.m = m;
    S.nf = nf;
    S.mc = m;
    S.nc = nf;
    S.prm = *prm;
    S.form = form;
    S.pc = pc;
    S.s = s;
    if (fabs(prm->kappa - nf->kappa) > 1e-12 * (1.0 + prm->kappa))
        return set_error(PB_EINVAL, "near field was built for kappa=%g, params say %g", nf->kappa, prm->kappa);
    double alpha = o ? o->alpha : 0.0, beta = o ? o->beta : 0.0;
    PB_TRY(system_blockop(prm, form, alpha, beta, &S.A));
    if (pc < PB_PC_NONE || pc > PB_PC_SCALED_CALDERON_EXT) return set_error(PB_EINVAL, "unknown preconditioner %d", pc);
    if (pc >= PB_PC_CALDERON_FULL) {
        if (form != PB_PMCHWT_INT && form != PB_PMCHWT_EXT)
            return set_error(PB_EINVAL, "Calderon preconditioners apply to the PMCHWT formulations");
        if (pc == PB_PC_CALDERON_FULL) S.C = S.A;
        else {
            int which = (pc == PB_PC_CALDERON_INT || pc == PB_PC_SCALED_CALDERON_INT) ? 0 : 1;
            PB_TRY(calderon_blockop(prm, form, which, &S.C));
            if (pc >= PB_PC_SCALED_CALDERON_INT) {
                half_calderon_scaling(prm, form, which, &S.sa, &S.sb);
                if (o && o->pc_a > 0.0 && o->pc_b > 0.0) { S.sa = o->pc_a; S.sb = o->pc_b; }
            }
        }
    }
    if (pc == PB_PC_SCALED_MASS) {
        // Juffer choice a = 1 + eps_ext/eps_int, b = 1 + eps_int/eps_ext (paper, after eq. prec:mass:scaled)
        S.sa = 1.0 + prm->eps_ext / prm->eps_int;
        S.sb = 1.0 + prm->eps_int / prm->eps_ext;
        if (o && o->pc_a > 0.0 && o->pc_b > 0.0) { S.sa = o->pc_a; S.sb = o->pc_b; }
    }
    const int64_t nv = m->nv, n2 = 2 * nv;
    PB_TRY(ws_reserve(const_cast<pb_mesh*>(m)->ws_vec, sizeof(double) * (4 * nv + 6 * n2)));
    double* p = (double*)m->ws_vec.ptr;
    S.bdiag = p; p += 4 * nv;
    S.t1 = p; p += n2;
    S.t2 = p; p += n2;
    S.t3 = p; p += n2;
    S.cheb = p;
    if (pc == PB_PC_BLOCK_DIAG) {
        k_block_diag_setup<<<nb(nv), 256, 0, s>>>(nv, nf->diag, S.A, S.bdiag);
        ::pb::count_launch();
    }
    PB_CUDA(cudaGetLastError());
    return PB_OK;
}

int check_status(const pb_mesh* m, cudaStream_t s) {
    int* status = m->status;
    int h = 0;
    PB_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    PB_CUDA(cudaStreamSynchronize(s));
    if (h != 0) {
        PB_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
        return set_error(PB_ETIMEOUT, "a bounded device wait gave up (status %d)", h);
    }
    return PB_OK;
}

// ---------------------------------------------- step-wise GMRES
void gm_norm2(GmresWork& G, const double* w, double* dst, cudaStream_t s) { dots(G, w, 1, w, dst, 0, s); }

int gm_begin(GmresWork& G, const double* w, const double* n2, cudaStream_t s) {
    const int ldh = G.mmax + 1;
    PB_CUDA(cudaMemsetAsync(G.H, 0, sizeof(double) * (size_t)ldh * G.mmax, s));
    PB_CUDA(cudaMemsetAsync(G.g, 0, sizeof(double) * (G.mmax + 2), s));
    k_gm_begin<<<1, 1, 0, s>>>(n2, G.g, G.res + 4, G.jdev);
    ::pb::count_launch();
    k_normalize0<<<nb(G.n), 256, 0, s>>>(G.n, w, n2, G.V, G.vin);
    ::pb::count_launch();
    PB_CUDA(cudaGetLastError());
    return PB_OK;
}

// Classical Gram-Schmidt applied twice (the second pass's coefficients are
// added to the first), normalisation and the Givens update of column j.
int gm_step(GmresWork& G, double* w, double* res_out, cudaStream_t s) {
    const int64_t n = G.n;
    const int ldh = G.mmax + 1;
    const int nchunk = (int)((n + DOT_CHUNK - 1) / DOT_CHUNK);
    const dim3 grid(nchunk, std::min(DOT_KY, G.mmax + 1));
    const unsigned kb = (unsigned)((G.mmax + 1 + 127) / 128);
    // algorithmic bytes at step j: the dots read V[0..j] and w once ((j + 2) n
    // doubles); the update reads V[0..j] and w and writes w ((j + 3) n doubles)
    const double nb8 = 8.0 * (double)n;
    for (int pass = 0; pass < 2; ++pass) {
        {
            Timer tm(G.ctx, PB_KERNEL_KRYLOV, s, nb8, 1.0, nb8);
            k_dots_j<<<grid, DOT_THREADS, 0, s>>>(n, G.V, w, G.part, nchunk, G.jdev);
            tm.stop();
        }
        k_dots_finish_j<<<kb, 128, 0, s>>>(nchunk, G.part, G.H, ldh, G.y, G.jdev, pass);
        {
            Timer tm(G.ctx, PB_KERNEL_KRYLOV, s, 2.0 * nb8, 1.0, nb8);
            k_vh_j<<<nb(n), 256, 0, s>>>(n, G.V, G.H, ldh, G.y, G.jdev, pass, w);
            tm.stop();
        }
        ::pb::count_launch(3);
    }
    k_dots<<<dim3(nchunk, 1), DOT_THREADS, 0, s>>>(n, w, n, w, G.part, nchunk);  // ||w||^2 partials
    k_hcol_j<<<1, 128, 0, s>>>(nchunk, G.part, G.H, ldh, G.y, G.jdev);
    k_normalize_j<<<nb(n), 256, 0, s>>>(n, w, G.H, ldh, G.jdev, G.V, G.vin);
    k_givens_j<<<1, 1, 0, s>>>(G.H, ldh, G.cs, G.sn, G.g, G.res + 4, res_out, G.jdev);
    ::pb::count_launch(4);
    PB_CUDA(cudaGetLastError());
    return PB_OK;
}

int gm_finish(GmresWork& G, int k, double* x, cudaStream_t s) {
    if (k <= 0) return PB_OK;
    k_backsolve<<<1, 1, 0, s>>>(k, G.H, G.mmax + 1, G.g, G.y);
    ::pb::count_launch();
    k_vh<<<nb(G.n), 256, 0, s>>>(G.n, k, G.V, G.n, G.y, 1.0, x);
    ::pb::count_launch();
    PB_CUDA(cudaGetLastError());
    return PB_OK;
}

int calderon_pre(Solver& S, int prec, const double* x) {
    return mass_solve(S.m, S.nf, x, S.t1, S.cheb, cheb_count(S, prec), S.s);
}

int calderon_post(Solver& S, int prec, double* y) {
    PB_TRY(mass_solve(S.m, S.nf, S.t2, y, S.cheb, cheb_count(S, prec), S.s));
    if (S.sa != 1.0 || S.sb != 1.0) {
        k_scale_halves<<<nb(2 * S.m->nv), 256, 0, S.s>>>(S.m->nv, 1.0 / S.sa, 1.0 / S.sb, y);
        ::pb::count_launch();
    }
    PB_CUDA(cudaGetLastError());
    return PB_OK;
}

void vec_sub(int64_t n, const double* a, const double* b, double* y, cudaStream_t s) {
    k_sub<<<nb(n), 256, 0, s>>>(n, a, b, y);
    ::pb::count_launch();
}
void vec_add(int64_t n, const double* a, double* y, cudaStream_t s) {
    k_add_inplace<<<nb(n), 256, 0, s>>>(n, a, y);
    ::pb::count_launch();
}

static int solve_body(pb_ctx* ctx, const pb_mesh* m, const pb_near* nf, const pb_params* prm, int form, int pc,
                      const pb_solve_opts* o, int nrhs, const double* b, double* x, pb_solve_info* info,
                      cudaStream_t s, Solver& S, const pb_mesh* mc, const pb_near* nc);

// The solve runs on a stream of its own, ordered after the caller's stream
// and before what the caller queues next: CUDA graphs cannot be captured on
// the legacy default stream.
static int solve_impl(pb_ctx* ctx, const pb_mesh* m, const pb_near* nf, const pb_params* prm, int form, int pc,
                      const pb_solve_opts* o, const double* b, double* x, pb_solve_info* info, cudaStream_t caller,
                      const pb_mesh* mc = nullptr, const pb_near* nc = nullptr, int nrhs = 1) {
    pb_solve_opts d = {1e-6, 500, 0, PB_F64, 1e-4, 20, 0, 0, 0, 0};
    if (!o) o = &d;
    if (!(o->tol > 0.0) || o->max_it < 1) return set_error(PB_EINVAL, "need tol > 0 and max_it >= 1");
    if (o->precision != PB_F64 && o->precision != PB_MIXED) return set_error(PB_EINVAL, "precision must be PB_F64 or PB_MIXED");
    cudaStream_t s = nullptr;
    cudaEvent_t fence = nullptr;
    PB_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    if (cudaEventCreateWithFlags(&fence, cudaEventDisableTiming) != cudaSuccess) {
        cudaStreamDestroy(s);
        return set_error(PB_ECUDA, "cudaEventCreate failed");
    }
    cudaEventRecord(fence, caller);
    cudaStreamWaitEvent(s, fence, 0);
    Solver S;
    int rc = solve_body(ctx, m, nf, prm, form, pc, o, nrhs, b, x, info, s, S, mc, nc);
    solver_release(S);
    cudaEventRecord(fence, s);
    cudaStreamWaitEvent(caller, fence, 0);
    cudaEventDestroy(fence);
    cudaStreamDestroy(s);
    return rc;
}

static int solve_one(const pb_mesh* m, const pb_near* nf, const pb_solve_opts* o, const double* b, double* x,
                     pb_solve_info* info, cudaStream_t s, Solver& S, GmresWork& G, int mmax);

// Solver set up once; the right-hand sides one after the other with the same
// Krylov workspace and the same captured iteration graphs.
static int solve_body(pb_ctx* ctx, const pb_mesh* m, const pb_near* nf, const pb_params* prm, int form, int pc,
                      const pb_solve_opts* o, int nrhs, const double* b, double* x, pb_solve_info* info,
                      cudaStream_t s, Solver& S, const pb_mesh* mc, const pb_near* nc) {
    PB_TRY(setup_solver(S, m, nf, prm, form, pc, o, s));
    if (mc) {
        S.mc = mc;
        S.nc = nc;
    }
    S.graphs = ctx->graphs != 0;
    const int64_t n2 = 2 * m->nv;
    int mmax = o->restart > 0 ? std::min(o->restart, o->max_it) : o->max_it;
    GmresWork G;
    PB_TRY(gmres_alloc(G, n2, mmax));
    G.ctx = ctx;
    int worst = PB_OK;
    for (int k = 0; k < nrhs; ++k) {
        const int rc = solve_one(m, nf, o, b + (size_t)k * n2, x + (size_t)k * n2, info ? info + k : nullptr, s, S,
                                 G, mmax);
        if (rc != PB_OK && rc != PB_ENOCONV) {
            gmres_free(G);
            return rc;
        }
        if (rc != PB_OK) worst = rc;
    }
    gmres_free(G);
    if (worst != PB_OK && nrhs > 1)
        set_error(worst, "GMRES did not reach tol %g for every right-hand side (see the infos)", o->tol);
    return worst;
}

static int solve_one(const pb_mesh* m, const pb_near* nf, const pb_solve_opts* o, const double* b, double* x,
                     pb_solve_info* info, cudaStream_t s, Solver& S, GmresWork& G, int mmax) {
    const int64_t n2 = 2 * m->nv;
    const int applies0 = S.applies;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    int rc = PB_OK, total_it = 0, outer = 0;
    double rel = 0.0;
    PB_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n2, s));
    if (o->precision == PB_F64) {
        // unrestarted, or restarted cycles when restart < max_it
        double beta0 = 0.0;
        while (rc == PB_OK && total_it < o->max_it) {
            int it = 0;
            double res = 0.0, beta = 0.0;
            rc = gmres(S, G, PB_F64, b, x, outer == 0, o->tol, beta0, std::min(mmax, o->max_it - total_it), &it,
                       &res, &beta);
            if (outer == 0) beta0 = beta;
            total_it += it;
            rel = res;
            ++outer;
            if (rc != PB_OK || rel <= o->tol || it == 0 || beta0 == 0.0) break;
        }
    } else {
        // Iterative refinement. Outer residual: split-coordinate FP32 pair sums
        // accumulated in FP64 per source tile plus the FP64 near field. Inner:
        // GMRES (FP64 Arnoldi) on A d = r with the FP32 operator.
        PhaseTrace tr("mixed");
        double* rr = nullptr;
        rc = dev_alloc((void**)&rr, sizeof(double) * 2 * n2);
        if (rc == PB_OK) {
            double* dd = rr + n2;
            double bnorm = 0.0, inner_last = 1.0;
            for (outer = 0; outer < std::max(1, o->max_outer) && rc == PB_OK; ++outer) {
                int it = 0;
                double res = 0.0, beta = 0.0;
                if (outer == 0) {
                    PB_CUDA(cudaMemcpyAsync(rr, b, sizeof(double) * n2, cudaMemcpyDeviceToDevice, s));
                } else {
                    const double* ca = nullptr;
                    rc = solver_comb(S, false, &ca);
                    if (rc == PB_OK) rc = apply_blockop(m, nf, S.A, PB_F32_ACCURATE, x, S.t3, s, ca);
                    if (rc != PB_OK) break;
                    S.applies++;
                    k_sub<<<nb(n2), 256, 0, s>>>(n2, b, S.t3, rr); ::pb::count_launch();
                }
                tr.lap("outer_residual");
                // ||P^-1 r|| with the accurate operator (no iterations)
                rc = gmres(S, G, PB_F32_ACCURATE, rr, dd, true, 0.0, 0.0, 0, &it, &res, &beta);
                if (rc != PB_OK) break;
                tr.lap("outer_norm");
                if (outer == 0) bnorm = beta;
                double prev = rel;
                rel = bnorm > 0.0 ? beta / bnorm : 0.0;
                tr.note("outer_rel", rel);
                if (rel <= o->tol) break;
                const double inner = refine_inner_tol(outer, rel, prev, inner_last, o->tol, o->inner_tol);
                if (inner < 0.0) break;  // the outer residual no longer falls: its own accuracy is reached
                inner_last = inner;
                PB_CUDA(cudaMemsetAsync(dd, 0, sizeof(double) * n2, s));
                rc = gmres(S, G, PB_F32, rr, dd, true, inner, 0.0, o->max_it, &it, &res, &beta);
                total_it += it;
                if (rc != PB_OK) break;
                tr.lap("inner_gmres");
                k_add_inplace<<<nb(n2), 256, 0, s>>>(n2, dd, x); ::pb::count_launch();
            }
            cudaFree(rr);
        }
    }
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == PB_OK) rc = check_status(m, s);
    if (rc == PB_OK && !(rel <= o->tol)) rc = set_error(PB_ENOCONV, "GMRES did not reach tol %g (residual %g after %d "
                                                        "iterations)", o->tol, rel, total_it);
    if (info) {
        info->status = rc;
        info->iters = total_it;
        info->outer_iters = outer;
        info->system_applies = S.applies - applies0;
        info->rel_residual = rel;
        info->time_ms = ms;
    }
    return rc;
}

}  // namespace pb

using namespace pb;

static int apply_args_ok(pb_ctx* ctx, const pb_mesh* m, const pb_near* nf, const void* x, const void* y) {
    if (!ctx || !m || !nf || !x || !y) return set_error(PB_EINVAL, "NULL argument");
    if (nf->mesh != m) return set_error(PB_EINVAL, "near field belongs to another mesh");
    return PB_OK;
}

extern "C" int pb_op_apply(pb_ctx* ctx, const pb_mesh* m, const pb_near* nf, int op, int kernel, int prec,
                           const double* x, double* y, void* stream) {
    PB_TRY(apply_args_ok(ctx, m, nf, x, y));
    if (op < PB_OP_V || op > PB_OP_M) return set_error(PB_EINVAL, "unknown operator %d", op);
    if (kernel != PB_LAPLACE && kernel != PB_YUKAWA) return set_error(PB_EINVAL, "unknown kernel %d", kernel);
    cudaStream_t s = (cudaStream_t)stream;
    BlockOp B;
    memset(&B, 0, sizeof(B));
    bool lap = kernel == PB_LAPLACE;
    int o, col;
    switch (op) {
        case PB_OP_V: o = lap ? O_VL : O_VY; col = 1; break;
        case PB_OP_K: o = lap ? O_KL : O_KY; col = 0; break;
        case PB_OP_T: o = lap ? O_TL : O_TY; col = 1; break;
        case PB_OP_D: o = lap ? O_DL : O_DY; col = 0; break;
        default: o = O_M; col = 0; break;
    }
    B.c[0][col][o] = 1.0;
    const int64_t nv = m->nv;
    PB_TRY(ws_reserve(const_cast<pb_mesh*>(m)->ws_vec, sizeof(double) * (4 * nv + 12 * nv)));
    double* in = (double*)m->ws_vec.ptr + 4 * nv;  // [u; v]
    double* out = in + 2 * nv;
    PB_CUDA(cudaMemsetAsync(in, 0, sizeof(double) * 2 * nv, s));
    PB_CUDA(cudaMemcpyAsync(in + col * nv, x, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
    PB_TRY(apply_blockop(m, nf, B, prec, in, out, s));
    PB_CUDA(cudaMemcpyAsync(y, out, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
    return PB_OK;
}

extern "C" int pb_system_apply(pb_ctx* ctx, const pb_mesh* m, const pb_near* nf, const pb_params* prm, int form,
                               double alpha, double beta, int prec, const double* x, double* y, void* stream) {
    PB_TRY(apply_args_ok(ctx, m, nf, x, y));
    if (x == y) return set_error(PB_EINVAL, "x and y must not overlap");
    BlockOp B;
    PB_TRY(system_blockop(prm, form, alpha, beta, &B));
    return apply_blockop(m, nf, B, prec, x, y, (cudaStream_t)stream);
}

extern "C" int pb_solve(pb_ctx* ctx, const pb_mesh* m, const pb_near* nf, const pb_params* prm, int form, int pc,
                        const pb_solve_opts* opts, const double* rhs, double* x, pb_solve_info* info, void* stream) {
    PB_TRY(apply_args_ok(ctx, m, nf, rhs, x));
    if (!prm) return set_error(PB_EINVAL, "NULL params");
    PB_CUDA(cudaSetDevice(ctx->device));
    return solve_impl(ctx, m, nf, prm, form, pc, opts, rhs, x, info, (cudaStream_t)stream);
}

extern "C" int pb_precond_apply(pb_ctx* ctx, const pb_mesh* m, const pb_near* nf, const pb_params* prm, int form,
                                int pc, const pb_solve_opts* opts, int prec, const double* x, double* y,
                                void* stream) {
    PB_TRY(apply_args_ok(ctx, m, nf, x, y));
    if (!prm) return set_error(PB_EINVAL, "NULL params");
    if (x == y) return set_error(PB_EINVAL, "x and y must not overlap");
    if (prec != PB_F64 && prec != PB_F32) return set_error(PB_EINVAL, "precision must be PB_F64 or PB_F32");
    PB_CUDA(cudaSetDevice(ctx->device));
    Solver S;
    PB_TRY(setup_solver(S, m, nf, prm, form, pc, opts, (cudaStream_t)stream));
    const int rc = apply_prec(S, prec, x, y);
    solver_release(S);
    return rc;
}

// Several right-hand sides of one system (one charge set each, e.g. the
// protonation states of a pKa calculation): one solver set-up, one Krylov
// workspace and one set of captured iteration graphs for all of them.
extern "C" int pb_solve_many(pb_ctx* ctx, const pb_mesh* m, const pb_near* nf, const pb_params* prm, int form, int pc,
                             const pb_solve_opts* opts, int nrhs, const double* rhs, double* x, pb_solve_info* info,
                             void* stream) {
    PB_TRY(apply_args_ok(ctx, m, nf, rhs, x));
    if (!prm) return set_error(PB_EINVAL, "NULL params");
    if (nrhs < 1) return set_error(PB_EINVAL, "pb_solve_many: need nrhs >= 1");
    PB_CUDA(cudaSetDevice(ctx->device));
    return solve_impl(ctx, m, nf, prm, form, pc, opts, rhs, x, info, (cudaStream_t)stream, nullptr, nullptr, nrhs);
}

// Fast Calderon (paper, "Fast Calderon preconditioning"): the preconditioner's
// operator from a second plan of the same surface.
extern "C" int pb_solve_pc(pb_ctx* ctx, const pb_mesh* m, const pb_near* nf, const pb_mesh* mc, const pb_near* nc,
                           const pb_params* prm, int form, int pc, const pb_solve_opts* opts, const double* rhs,
                           double* x, pb_solve_info* info, void* stream) {
    PB_TRY(apply_args_ok(ctx, m, nf, rhs, x));
    if (!prm || !mc || !nc) return set_error(PB_EINVAL, "NULL argument");
    if (nc->mesh != mc) return set_error(PB_EINVAL, "preconditioner near field belongs to another mesh");
    if (mc->nv != m->nv || mc->nt != m->nt)
        return set_error(PB_EINVAL, "preconditioner mesh differs from the system's (%lld/%lld vs %lld/%lld)",
                         (long long)mc->nv, (long long)mc->nt, (long long)m->nv, (long long)m->nt);
    if (pc < PB_PC_CALDERON_FULL) return set_error(PB_EINVAL, "pb_solve_pc needs a Calderon preconditioner");
    if (fabs(nc->kappa - nf->kappa) > 1e-12 * (1.0 + nf->kappa))
        return set_error(PB_EINVAL, "the two near fields were built for different kappa");
    PB_CUDA(cudaSetDevice(ctx->device));
    return solve_impl(ctx, m, nf, prm, form, pc, opts, rhs, x, info, (cudaStream_t)stream, mc, nc);
}
