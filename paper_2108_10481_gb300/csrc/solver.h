// Solver pieces shared by pb_solve (solve.cu) and the request server (serve.cu).
#pragma once

#include "internal.h"
#include "refine.h"

#include <algorithm>

namespace pb {

struct Solver {
    const pb_mesh* m;
    const pb_near* nf;
    const pb_mesh* mc = nullptr;  // the Calderon preconditioner's operator (fast Calderon: another plan)
    const pb_near* nc = nullptr;
    pb_params prm;
    int form, pc;
    BlockOp A, C;
    double sa = 1.0, sb = 1.0;  // scaling of the two halves after the preconditioner
    double* bdiag = nullptr;    // 4 nv
    double* t1 = nullptr;       // 2 nv each
    double* t2 = nullptr;
    double* t3 = nullptr;
    double* cheb = nullptr;     // 3 x 2 nv
    int cheb_iters = 34;
    int applies = 0;
    cudaStream_t s;
    bool graphs = false;        // replay iterations from CUDA graphs
    StepGraph step[4];          // GMRES iteration body, by operator precision
    // the near values combined for A and for C (4 nnz doubles, then 4 nnz floats each),
    // made on first use and kept for the solve
    double* combA = nullptr;
    double* combC = nullptr;
};
// the combined near values of the system (calderon = false) or of the Calderon operator
int solver_comb(Solver& S, bool calderon, const double** out);
void solver_release(Solver& S);

struct GmresWork {
    double* V = nullptr;     // (m+1) x n
    double* w = nullptr;     // n
    double* H = nullptr;     // (m+1) x m, column-major
    double* cs = nullptr;
    double* sn = nullptr;
    double* g = nullptr;     // m + 1
    double* y = nullptr;     // m
    double* part = nullptr;  // (m+1) x nchunk
    double* res = nullptr;   // res[0..1] estimates, res[4] beta (device)
    double* vin = nullptr;   // n: copy of V[j], the operator's input
    int* jdev = nullptr;     // the iteration index j, kept on the device
    int mmax = 0;
    pb_ctx* ctx = nullptr;   // profiled context of the Gram-Schmidt kernels (null: not profiled)
    int64_t n = 0;
    void* block = nullptr;
};


int setup_solver(Solver& S, const pb_mesh* m, const pb_near* nf, const pb_params* prm, int form, int pc,
                 const pb_solve_opts* o, cudaStream_t s);
int apply_prec(Solver& S, int prec, const double* x, double* y);
int gmres_alloc(GmresWork& G, int64_t n, int mmax);
void gmres_free(GmresWork& G);
void dots(GmresWork& G, const double* V, int nk, const double* w, double* out, int accumulate, cudaStream_t s);
int check_status(const pb_mesh* m, cudaStream_t s);

// step-wise GMRES: every scalar, the iteration index included, stays on the
// device, so that one iteration is the same launch sequence for every j
void gm_norm2(GmresWork& G, const double* w, double* dst, cudaStream_t s);
// g = beta e1 with beta = sqrt(n2[0]); V[0] = vin = w / beta; j = 0
int gm_begin(GmresWork& G, const double* w, const double* n2, cudaStream_t s);
// w = P^-1 A V[j]: orthogonalise, append V[j+1] (and vin), rotate column j;
// res_out[0] = |g[j+1]| / beta, res_out[1] = the new diagonal; j += 1
int gm_step(GmresWork& G, double* w, double* res_out, cudaStream_t s);
int gm_finish(GmresWork& G, int k, double* x, cudaStream_t s);
// Calderon preconditioner split around its operator application (t1 -> t2)
int calderon_pre(Solver& S, int prec, const double* x);
int calderon_post(Solver& S, int prec, double* y);
void vec_sub(int64_t n, const double* a, const double* b, double* y, cudaStream_t s);
void vec_add(int64_t n, const double* a, double* y, cudaStream_t s);

}  // namespace pb
