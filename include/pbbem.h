/*
 * pbbem.h - C ABI of the GB300 boundary-element Poisson-Boltzmann library.
 *
 * Problem (arxiv 2108.10481, eq. poissonboltzmann): a closed molecular
 * surface Gamma separates an interior region (permittivity eps_int, point
 * charges q_j at x_j) from a solvent (permittivity eps_ext, inverse Debye
 * length kappa). The library discretises the interior Laplace and exterior
 * Yukawa boundary operators (paper eq. layer_potentials: single layer V,
 * double layer K, adjoint double layer T, hypersingular D) with continuous
 * piecewise-linear (P1) Galerkin elements on a triangle mesh (paper,
 * "Numerical discretization": one unknown per vertex and trace), solves one
 * of the paper's boundary integral formulations with preconditioned GMRES and
 * returns the polar solvation energy (paper eq. dG).
 *
 * Conventions
 *   - Every function returns an int status: PB_OK (0) or a negative PB_E*
 *     code. On error a message is stored per thread and pb_last_error()
 *     returns it. No function aborts, traps or exits the process.
 *   - "device" pointers are CUDA device addresses on the context's device,
 *     owned by the caller (e.g. torch tensors); "host" pointers are ordinary
 *     CPU memory. Arrays are dense, row-major, 64-bit floats unless stated.
 *   - Unknown vectors have 2*N_v entries: x = [u; v] with u the Dirichlet and
 *     v the Neumann trace coefficients (P1, one per vertex) on the side the
 *     formulation solves for (interior or exterior, paper eqs.
 *     bie:dirichlet:int ... bie:lu:ext).
 *   - stream: a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Compute calls enqueue work on it; calls that return host
 *     scalars (pb_energy, pb_solve's info) synchronise it.
 *   - Handles (pb_ctx, pb_mesh, pb_near) are owned by the library and freed
 *     with their pb_free_* call. A handle may be used from one host thread at
 *     a time.
 *   - Units: lengths in Angstrom, charges in e; potentials in "paper units"
 *     (G = 1/(4 pi r), sources q/eps_int); energies additionally in kcal/mol.
 */
#ifndef PBBEM_H
#define PBBEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PB_OK 0
#define PB_EINVAL (-1)   /* bad argument (NULL handle, size, enum, pointer kind) */
#define PB_EMESH (-2)    /* mesh is not a closed, oriented, 2-manifold surface */
#define PB_ENOMEM (-3)   /* device or host allocation failed */
#define PB_ENOCONV (-4)  /* GMRES reached max_it before tol (best x returned) */
#define PB_ENUMERIC (-5) /* NaN or Inf met in a residual */
#define PB_ECUDA (-6)    /* a CUDA runtime call failed */
#define PB_ETIMEOUT (-7) /* a bounded device-side wait gave up */

/* ---- enumerations ------------------------------------------------------ */
/* operators of paper eq. layer_potentials, plus the mass matrix */
#define PB_OP_V 0
#define PB_OP_K 1
#define PB_OP_T 2
#define PB_OP_D 3
#define PB_OP_M 4
/* Green's functions (paper, "Boundary integral formulations"):
 * G_int = 1/(4 pi r), G_ext = exp(-kappa r)/(4 pi r) */
#define PB_LAPLACE 0
#define PB_YUKAWA 1
/* arithmetic of a far-field application */
#define PB_F64 0          /* FP64 everywhere */
#define PB_F32 1          /* FP32 pair sums and FP32 near field (inner solves) */
#define PB_F32_ACCURATE 2 /* FP32 pair arithmetic on split (hi+lo) coordinates with
                             FP64 accumulation per source tile, FP64 near field */
#define PB_MIXED 3        /* (pb_solve_opts.precision) FP32 inner GMRES inside FP64
                             iterative refinement */

/* formulations (paper, "Boundary integral formulations") */
#define PB_DIRECT_INT 0      /* eq. bie:dirichlet:int, unknowns interior */
#define PB_DIRECT_EXT 1      /* eq. bie:dirichlet:ext, unknowns exterior */
#define PB_DIRECT_INT_PERM 2 /* the same two rows swapped */
#define PB_DIRECT_EXT_PERM 3
#define PB_CFIE_INT 4        /* eq. bie:combined:int, alpha and beta from the opts */
#define PB_CFIE_EXT 5        /* eq. bie:combined:ext */
#define PB_PMCHWT_INT 6      /* eq. bie:pmchwt:int (alpha = beta = -1, as printed) */
#define PB_PMCHWT_EXT 7      /* eq. bie:pmchwt:ext */
#define PB_MULLER_INT 8      /* eq. bie:muller:int (alpha = beta = 1) */
#define PB_MULLER_EXT 9      /* eq. bie:muller:ext */
#define PB_JUFFER 10         /* eq. bie:juffer:int (alpha = eps_ext/eps_int, beta = 1/alpha) */
#define PB_LU 11             /* eq. bie:lu:ext (second row scaled by eps_int/eps_ext) */

/* preconditioners (paper, "Preconditioning") */
#define PB_PC_NONE 0
#define PB_PC_BLOCK_DIAG 1          /* per-DOF inverse of the diagonals of the four blocks */
#define PB_PC_MASS 2                /* eq. prec:mass */
#define PB_PC_SCALED_MASS 3         /* eq. prec:mass:scaled, (a, b) from the opts or the
                                       Juffer default a = 1+eps_ext/eps_int, b = 1+eps_int/eps_ext */
#define PB_PC_CALDERON_FULL 4       /* eqs. prec:calderon:int:full / ext:full (PMCHWT only) */
#define PB_PC_CALDERON_INT 5        /* interior half Calderon */
#define PB_PC_CALDERON_EXT 6        /* exterior half Calderon */
#define PB_PC_SCALED_CALDERON_INT 7 /* scaled mass on top of the interior half Calderon */
#define PB_PC_SCALED_CALDERON_EXT 8 /* ... of the exterior half Calderon */

typedef struct pb_ctx pb_ctx;
typedef struct pb_mesh pb_mesh;
typedef struct pb_near pb_near;

/* physical parameters (paper eq. poissonboltzmann) */
typedef struct {
    double eps_int; /* interior permittivity (> 0) */
    double eps_ext; /* solvent permittivity (> 0) */
    double kappa;   /* inverse Debye length, 1/Angstrom (>= 0) */
} pb_params;

/* quadrature plan: the discrete definition of every operator entry
 * (paper, Results: the orders of the regular and singular rules). A zeroed
 * struct is not a valid plan; {6, 4, 0.0, 6, 0, 0, 0} is the reference plan. */
typedef struct {
    int far_q; /* points of the symmetric triangle rule used on both triangles of
                  pairs that share no vertex: 1, 3 (degree 2) or 6 (degree 4) */
    int n_ss;  /* Gauss-Legendre points per dimension of the regularised [0,1]^4
                  rule for coincident, edge- and vertex-adjacent pairs (1..12) */
    double band_eta; /* distance band (0 = none, else in (0, 64]): pairs sharing no
                  vertex whose centroids are closer than band_eta times the sum
                  of their radii (largest centroid-vertex distance) take the
                  band rule instead of far_q; the far-field pair kernel then
                  runs with far_q and the near field adds the difference */
    int band_q; /* band rule (3 or 6, finer than far_q; 0 means 6). With a band,
                  the right-hand side and the energy use the band rule. */
    int n_ss_coin; /* Gauss points per dimension of the singular rule for each */
    int n_ss_edge; /* class of adjacent pair: coincident, edge-adjacent, vertex- */
    int n_ss_vert; /* adjacent (1..12; 0 means n_ss). The paper states one order. */
} pb_quad_plan;

/* memory kind of pb_mesh_load's inputs */
#define PB_MEM_HOST 0
#define PB_MEM_DEVICE 1

typedef struct {
    double tol;        /* relative left-preconditioned residual target */
    int max_it;        /* GMRES iterations (per refinement sweep for PB_MIXED) */
    int restart;       /* 0 = unrestarted (basis of max_it vectors) */
    int precision;     /* PB_F64 or PB_MIXED */
    double inner_tol;  /* PB_MIXED: smallest relative tolerance an inner solve asks for */
    int max_outer;     /* PB_MIXED: refinement sweeps at most */
    double alpha;      /* PB_CFIE_INT / PB_CFIE_EXT coefficients */
    double beta;
    double pc_a;       /* scaled-mass constants; 0 = the paper's choice */
    double pc_b;
} pb_solve_opts;

typedef struct {
    int status;          /* same as the return code */
    int iters;           /* total GMRES iterations (all sweeps) */
    int outer_iters;     /* refinement sweeps (1 for PB_F64) */
    int system_applies;  /* far-field system applications */
    double rel_residual; /* final ||P^-1 (b - A x)|| / ||P^-1 b|| (FP64 outer estimate) */
    double time_ms;      /* device time of the solve */
} pb_solve_info;

/* ---- context ------------------------------------------------------------ */
/* Create a context on CUDA device `device`. Returns PB_ECUDA if the device
 * cannot be used, PB_EINVAL if out is NULL. */
int pb_init(int device, pb_ctx** out);
/* Free a context (NULL is allowed). Meshes and near fields must be freed first. */
int pb_free_ctx(pb_ctx* ctx);
/* Message of the last error on this thread ("" if none). Never NULL. */
const char* pb_last_error(void);
/* Library version string, e.g. "pbbem 0.1 sm_103a". */
const char* pb_version(void);

/* ---- a1: mesh ingest ---------------------------------------------------- */
/* Copy in and validate a triangle mesh (paper, "Numerical discretization":
 * P1 elements on a triangular surface mesh; eq. poissonboltzmann: the
 * interface Gamma with outward normal n).
 *   verts: n_verts x 3 doubles; tris: n_tris x 3 int32 vertex indices listed
 *   counter-clockwise seen from outside; mem: PB_MEM_HOST or PB_MEM_DEVICE.
 * Checks: indices in range, no zero-area triangle, every edge shared by
 * exactly two triangles with opposite orientations (closed, oriented
 * 2-manifold), positive enclosed volume; else PB_EMESH. Builds the
 * quadrature points of `plan` (NULL = {6, 4}), the vertex->triangle map, the
 * adjacent triangle pairs and the vertex-pair pattern of the near field.
 * The library owns *out; free with pb_free_mesh. */
int pb_mesh_load(pb_ctx* ctx, const double* verts, int64_t n_verts, const int32_t* tris,
                 int64_t n_tris, const pb_quad_plan* plan, int mem, pb_mesh** out);
int pb_free_mesh(pb_mesh* mesh);
/* Sizes of a loaded mesh: out[0..5] = N_v, N_t, quadrature points, near
 * nonzeros per operator, adjacent triangle pairs, device bytes held. */
int pb_mesh_info(const pb_mesh* mesh, int64_t out[6]);

/* ---- a2: near field ----------------------------------------------------- */
/* FP64 device build of the singular near field for Yukawa parameter kappa:
 * for every pair of triangles sharing a vertex, the regularised-quadrature
 * local blocks of V, K, D (Laplace and Yukawa) minus the same blocks by the
 * far rule, summed into a vertex-pair CSR (T by transposition, M exact), and
 * the full operator diagonals. Reusable for any charges with the same kappa.
 * The library owns *out; free with pb_free_near. */
int pb_near_build(pb_ctx* ctx, const pb_mesh* mesh, double kappa, pb_near** out, void* stream);
int pb_free_near(pb_near* near);

/* ---- a3 + a4 + a5: operator application --------------------------------- */
/* y = A x for one Galerkin operator (N_v -> N_v): op in PB_OP_V..PB_OP_M,
 * kernel PB_LAPLACE or PB_YUKAWA (ignored for PB_OP_M), prec PB_F64, PB_F32
 * or PB_F32_ACCURATE. x and y are device arrays of N_v doubles and must not
 * overlap. The near field must have been built for the kappa wanted. */
int pb_op_apply(pb_ctx* ctx, const pb_mesh* mesh, const pb_near* near, int op, int kernel,
                int prec, const double* x, double* y, void* stream);
/* y = A x for the 2x2 weak-form system of a formulation (PB_DIRECT_INT ...
 * PB_LU; alpha/beta used by the CFIE forms only). x, y: device, 2*N_v. */
int pb_system_apply(pb_ctx* ctx, const pb_mesh* mesh, const pb_near* near, const pb_params* prm,
                    int form, double alpha, double beta, int prec, const double* x, double* y,
                    void* stream);

/* Allocation-free FP32 system application (the paper has no counterpart: it
 * exists for callers that cannot call cudaMalloc). It computes the FP32
 * system application of pb_system_apply(..., PB_F32, ...) - the same sources,
 * per-triangle reduction, gather and FP32 near field - but always with the
 * direct scalar FP32 pair kernel (k_pair32, at most 4 source splits), and it
 * keeps every temporary in one file-scope device array of 16 MiB that each GPU
 * loading the library holds until the process exits; it calls no cudaMalloc,
 * cudaFree or other allocating routine. Its result therefore differs from
 * pb_system_apply's by FP32 rounding in another summation order (the packed
 * kernel or another split count; about 1e-6 relative), and by the treecode's
 * approximation (about 1e-5) where pb_system_apply uses the treecode (meshes
 * with at least pb_set_treecode's min_points far-rule points). The mesh and
 * near field must come from ctx (else PB_EINVAL). The callers it is for: processes
 * whose device memory belongs to another allocator that reserves it up front
 * (a raw cudaMalloc would fail or take memory that allocator counts on), and
 * latency-bound loops that cannot afford the device-wide synchronisation that
 * cudaMalloc and cudaFree bring.
 *   - Limit: meshes whose temporaries fit in 16 MiB (about 9,000 triangles
 *     with the 6-point rule); larger meshes get PB_EINVAL with the sizes.
 *   - The first call on a device, with that device current, looks up the
 *     array's device address once (cudaGetSymbolAddress); make that first call
 *     before any stream capture.
 *   - All calls share the one array and it keeps the last call's contents
 *     (each call writes every word it later reads, so nothing must start at
 *     zero). Calls that overlap on the GPU - on different streams, or from
 *     different threads - race on it and must not be issued.
 * x, y: device arrays of 2*N_v doubles that must not overlap; the caller owns
 * them. */
int pb_system_apply_noalloc(pb_ctx* ctx, const pb_mesh* mesh, const pb_near* near, const pb_params* prm,
                            int form, double alpha, double beta, const double* x, double* y, void* stream);

/* ---- a6: right-hand side ------------------------------------------------ */
/* rhs = the formulation's right-hand side built from the source projections
 * (paper eq. sources: phi_D = sum_j q_j/(4 pi eps_int |x - x_j|), phi_N its
 * normal derivative), tested against the P1 basis with the plan's reference
 * rule. xq (n_q x 3) and q (n_q) are device arrays; rhs is device, 2*N_v.
 * prec: PB_F64 (FP64 pair arithmetic) or PB_F32_ACCURATE (FP32 pair arithmetic
 * on split hi + lo coordinates relative to the mesh centre, FP32 sums over
 * tiles of 256 charges added in FP64: about 1e-7 relative, for the
 * mixed-precision path). */
int pb_rhs_charges(pb_ctx* ctx, const pb_mesh* mesh, const double* xq, const double* q, int64_t n_q,
                   const pb_params* prm, int form, double alpha, double beta, double* rhs, int prec,
                   void* stream);

/* ---- a7 + a8 + a9: preconditioned GMRES --------------------------------- */
/* Solve P^-1 A x = P^-1 rhs (paper, "Preconditioning": left preconditioning,
 * GMRES) from x = 0. opts NULL = {tol 1e-6, max_it 500, unrestarted, PB_F64}.
 * rhs and x are device arrays of 2*N_v. On PB_ENOCONV x holds the best
 * iterate and info (optional) is filled.
 * PB_MIXED: each sweep computes the residual r = rhs - A x with PB_F32_ACCURATE
 * applications and its preconditioned norm, stops once that is at most tol
 * relative to the right-hand side's, and otherwise solves A d = r with PB_F32
 * applications to min(0.1, max(inner_tol, tol / rel)) of the current relative
 * residual rel and adds d to x. After a sweep (from the second on) that did
 * not halve the residual the next one asks for 1e-3; a sweep that asked for 1e-3 (or inner_tol, if
 * larger) and still did not halve it ends the solve (PB_ENOCONV if above tol):
 * the split-coordinate residual's own accuracy, about 2e-8 relative on the
 * molecules, is then reached. */
int pb_solve(pb_ctx* ctx, const pb_mesh* mesh, const pb_near* near, const pb_params* prm, int form,
             int precond, const pb_solve_opts* opts, const double* rhs, double* x,
             pb_solve_info* info, void* stream);
/* pb_solve for nrhs right-hand sides of the same system (paper: fast solves
 * pay off for many right-hand sides, e.g. the charge sets of pKa
 * calculations): rhs and x hold nrhs vectors of 2*N_v one after another
 * (device), info (optional) nrhs records. The solver is set up once and the
 * Krylov workspace and captured iteration graphs serve every right-hand side.
 * Returns PB_ENOCONV when any did not converge (its info says which). */
int pb_solve_many(pb_ctx* ctx, const pb_mesh* mesh, const pb_near* near, const pb_params* prm, int form,
                  int precond, const pb_solve_opts* opts, int nrhs, const double* rhs, double* x,
                  pb_solve_info* info, void* stream);
/* pb_solve with the Calderon preconditioner's operator taken from a second
 * discretisation of the same surface (paper, "Fast Calderon preconditioning":
 * relaxed quadrature orders for the preconditioner only, e.g. the 1-point far
 * rule and 3 singular Gauss points; the solution is that of the system's own
 * plan). pc_mesh must be the same vertices and triangles loaded with another
 * plan (same counts, else PB_EINVAL) and pc_near its near field; precond must
 * be one of the Calderon preconditioners. Otherwise as pb_solve. */
int pb_solve_pc(pb_ctx* ctx, const pb_mesh* mesh, const pb_near* near, const pb_mesh* pc_mesh,
                const pb_near* pc_near, const pb_params* prm, int form, int precond, const pb_solve_opts* opts,
                const double* rhs, double* x, pb_solve_info* info, void* stream);

/* y = P^-1 x: the preconditioner of pb_solve for formulation `form` and
 * preconditioner `precond` (paper, "Preconditioning": block diagonal, mass,
 * scaled mass and the Calderon products, with the mass inverse by the same
 * Chebyshev iteration: 34 steps, 16 with prec = PB_F32, the count the FP32
 * inner iterations use), operator applications in precision prec (PB_F64 or
 * PB_F32). opts supplies alpha, beta (CFIE) and pc_a, pc_b (scalings; NULL =
 * defaults). x and y: device, 2*N_v, not overlapping. Used with
 * pb_system_apply to form P^-1 A for spectra (paper, eigenvalue figures). */
int pb_precond_apply(pb_ctx* ctx, const pb_mesh* mesh, const pb_near* near, const pb_params* prm, int form,
                     int precond, const pb_solve_opts* opts, int prec, const double* x, double* y, void* stream);

/* ---- a10: reaction potential and solvation energy ------------------------ */
/* phi_reac(x_j) = V_int[v_int](x_j) - K_int[u_int](x_j) (paper eq.
 * phireac_bie) from the solution x of formulation `form` (exterior forms are
 * converted by u_int = u_ext, v_int = (eps_ext/eps_int) v_ext), and
 * Delta G = 1/2 sum_j q_j phi_reac(x_j) (paper eq. dG), reduced in FP64.
 * xq, q device; dG_paper and dG_kcal host (either may be NULL); phi (device,
 * n_q, may be NULL) receives phi_reac. prec: PB_F64 or PB_F32_ACCURATE (the
 * point-charge pair sums in FP32 on split coordinates, FP32 sums over tiles
 * of 256 points added in FP64; the reduction over charges in FP64 either way). */
int pb_energy(pb_ctx* ctx, const pb_mesh* mesh, const double* x, int form, const double* xq,
              const double* q, int64_t n_q, const pb_params* prm, double* phi, double* dG_paper,
              double* dG_kcal, int prec, void* stream);

/* ---- whole path from host buffers --------------------------------------- */
/* One solve from host arrays: mesh load, near build, right-hand side, solve
 * and energy, freeing everything it made. verts/tris/xq/q are host arrays;
 * dG_kcal (host) receives the energy in kcal/mol. With opts->precision =
 * PB_MIXED the right-hand side and the energy take PB_F32_ACCURATE. */
int pb_solvation_energy(pb_ctx* ctx, const double* verts, int64_t n_verts, const int32_t* tris,
                        int64_t n_tris, const double* xq, const double* q, int64_t n_q,
                        const pb_params* prm, const pb_quad_plan* plan, int form, int precond,
                        const pb_solve_opts* opts, double* dG_kcal, pb_solve_info* info,
                        void* stream);

/* ---- a11: request server (continuous batching) --------------------------- */
/* Serving many molecules on one GPU. Not in the paper: its solves run one at
 * a time; this is the batched form of the same path (pb_mesh_load ...
 * pb_energy per request) with results equal to solving each request alone. */
typedef struct pb_server pb_server;

typedef struct {
    const double* verts;   /* host, n_verts x 3 (copied at submit) */
    int64_t n_verts;
    const int32_t* tris;   /* host, n_tris x 3, counter-clockwise seen from outside */
    int64_t n_tris;
    const double* xq;      /* host, n_q x 3 charge positions */
    const double* q;       /* host, n_q charges */
    int64_t n_q;
    pb_params params;
    int form;              /* PB_DIRECT_INT ... PB_LU */
    int precond;           /* PB_PC_* */
    pb_solve_opts opts;    /* tol, max_it, restart (Krylov basis size; 0 = max_it), precision, ... */
    pb_quad_plan plan;     /* {0, 0} = the default {6, 4} */
    uint64_t tag;          /* the caller's identifier, returned in the result */
} pb_request;

typedef struct {
    uint64_t tag;
    int status;            /* PB_OK, PB_ENOCONV (best iterate used), or the error of its setup */
    int iters;             /* GMRES iterations */
    int outer_iters;       /* refinement sweeps (1 for FP64) */
    double dG_kcal;        /* polar solvation energy */
    double dG_paper;
    double rel_residual;   /* final relative preconditioned residual */
    double latency_ms;     /* submit -> result */
    double queue_ms;       /* submit -> set up and ready to iterate */
} pb_result;

/* Create a server on ctx's device that keeps at most max_active requests
 * resident and admits a request only while the sum of the admitted requests'
 * device footprints (estimated from their sizes, Krylov basis included) stays
 * within hbm_budget_bytes. Starts one host thread for admission. */
int pb_server_create(pb_ctx* ctx, int64_t hbm_budget_bytes, int max_active, pb_server** out);
/* Stop the admission thread and free every resident request. */
int pb_server_destroy(pb_server* srv);
/* Queue a request (its arrays are copied). PB_ENOMEM if it alone exceeds the
 * budget, PB_EINVAL for a malformed request. Thread-safe. */
int pb_submit(pb_server* srv, const pb_request* req);
/* One scheduling step: move newly set-up requests into the active set and
 * advance every active request by one GMRES step, all their operator
 * applications in one batched pair-kernel launch per row mode; finished
 * requests compute their energy and release their memory. Returns at once
 * when nothing is active. Call from one thread. */
int pb_server_step(pb_server* srv, int* n_active, int* n_pending);
/* Move up to max finished results into out; *n_out = how many. Thread-safe. */
int pb_poll(pb_server* srv, pb_result* out, int max, int* n_out);

/* ---- a12: autotuner --------------------------------------------------------- */
/* Launch tuning of the FP32 far field (not in the paper: its software uses
 * fixed FMM and quadrature settings). */
typedef struct {
    int kernel;             /* chosen FP32 kernel: 1 scalar, 2 packed f32x2 */
    int shape;              /* launch shape of the packed kernel (0 = default) */
    int tile_records;       /* source records per TMA tile of the chosen launch */
    int stages;             /* its pipeline stages */
    int targets_per_thread; /* its targets per thread */
    int tiles_per_fp64_sum; /* split-coordinate variant: tiles whose FP32 sums go into FP64 at a time */
    double split_scale;     /* chosen multiplier of the wave-filling split count */
    double best_ms;         /* one FP32 system application with the choice */
    double default_ms;      /* ... with the untuned default (packed, shape 0, x1) */
} pb_tune_choice;
typedef struct {
    pb_tune_choice fast;     /* PB_F32 applications (FP32 tile sums) */
    pb_tune_choice accurate; /* PB_F32_ACCURATE applications (split coordinates, FP64 tile sums) */
} pb_tune_result;
/* Time every candidate launch of formulation `form`'s FP32 system application
 * on this mesh (fast and split-coordinate variants; the scalar kernel and the
 * packed kernel in each of its launch shapes - records per TMA tile 32, 64
 * or 128, 2 or 4 pipeline stages, 2 or 4 targets per thread, for the
 * split-coordinate variant 1, 2 or 4 tiles per FP64 addition - each with the
 * wave-filling split count x0.5, x1 and x2) and keep the fastest of each
 * variant in ctx for meshes of this size (same power-of-two bucket of
 * quadrature points). Later applications, solves and the server use it. out
 * may be NULL. The treecode is off while the candidates are timed (the choice
 * is the direct pair kernel's: PB_F32 applications of meshes that take the
 * treecode use it only when the treecode is switched off); the context must
 * not be in use by another host thread meanwhile. */
int pb_autotune(pb_ctx* ctx, const pb_mesh* mesh, const pb_near* near, const pb_params* prm, int form,
                pb_tune_result* out, void* stream);
/* Quadrature plan for a molecule: solve it (host arrays, like
 * pb_solvation_energy) with `reference` (NULL = {6, 4}) and with cheaper
 * plans, and return in out_plan the cheapest plan whose Delta G differs from
 * the reference one by at most tol_dG relative (the reference plan when none
 * does); *out_change (optional) = that difference. Candidates: first the
 * 3-point far rule with the reference's rule inside a distance band of 2, 3,
 * 4 and 6 radii (the first that qualifies is kept), then, one class at a
 * time (vertex-adjacent, edge-adjacent, coincident pairs), one Gauss point
 * fewer per dimension of that class's singular rule, each kept if the plan
 * still qualifies. */
int pb_autotune_plan(pb_ctx* ctx, const double* verts, int64_t n_verts, const int32_t* tris, int64_t n_tris,
                     const double* xq, const double* q, int64_t n_q, const pb_params* prm,
                     const pb_quad_plan* reference, int form, int precond, const pb_solve_opts* opts, double tol_dG,
                     pb_quad_plan* out_plan, double* out_change, void* stream);

/* ---- measurement ---------------------------------------------------------- */
/* kernel families timed by pb_profile */
#define PB_KERNEL_PAIR32 0          /* FP32 far-field pair kernel (inner solves) */
#define PB_KERNEL_PAIR32_ACCURATE 1 /* split-coordinate FP32 pair kernel (outer residuals) */
#define PB_KERNEL_PAIR64 2          /* FP64 pair kernel */
#define PB_KERNEL_NEAR_ADJ 3        /* FP64 regularised quadrature of edge- and vertex-adjacent pairs */
#define PB_KERNEL_NEAR_COIN 4       /* FP64 regularised quadrature of coincident pairs */
#define PB_KERNEL_NEAR_BAND 5       /* FP64 band-rule minus far-rule blocks of band pairs */
#define PB_KERNEL_TREE32 6          /* FP32 treecode evaluation (proxy and direct interactions) */
#define PB_KERNEL_SPMV 7            /* gather of the triangle sums + near-field SpMV (memory-bound) */
#define PB_KERNEL_CHEB 8            /* one Chebyshev step of the mass solve (memory-bound) */
#define PB_KERNEL_KRYLOV 9          /* Gram-Schmidt dots and updates of the Arnoldi step (memory-bound) */
#define PB_KERNEL_COUNT 10
/* For the pair kernels, "pairs" are target-source point pairs and "ops" FP32
 * (FP64 for PB_KERNEL_PAIR64) operations by the kernel's formula count; for
 * the near-field kernels, "pairs" are quadrature point pairs (kernel
 * evaluations) and "ops" FP64 flops by formula count (kernel evaluation and
 * accumulation into the local blocks, a fused multiply-add counted as two).
 * For the memory-bound families (SPMV, CHEB, KRYLOV) "pairs" and "ops" are
 * both the algorithmic bytes of the launches: every array element the launch
 * must read or write, counted once. */
/* enable (1) or disable (0) per-launch CUDA-event timing of the pair kernels
 * on their launching stream; either call resets the statistics. No effect on
 * results. */
int pb_profile(pb_ctx* ctx, int enable);
/* Statistics of one kernel family since pb_profile(ctx, 1): launches, summed
 * device time in ms, target-source point pairs, and FP32/FP64 pipe operations
 * by the kernel's formula count (operations per pair x pairs). Waits for the
 * recorded events. Any output pointer may be NULL. */
int pb_profile_read(pb_ctx* ctx, int kernel, int64_t* launches, double* total_ms, double* pairs, double* ops);
/* Failure detection self-test: run the pair kernels' bounded mbarrier wait on a
 * barrier that nothing completes, giving up after `polls` polls (1..2^24);
 * *status_out receives the status word the kernel wrote (PB_ETIMEOUT when the
 * wait ran out). The kernel returns normally and the context stays usable. */
int pb_selftest_wait(pb_ctx* ctx, int64_t polls, int* status_out);
/* Self-test of the exponential the FP64 near-field kernels use for the Yukawa
 * factor e^{-kappa r} (a table-driven e^x for x <= 0 after Tang, ACM TOMS
 * 15(2), 1989): y[i] = e^{x[i]} for the n device doubles x (each <= 0; 0 is
 * returned below -700), on `stream` (NULL: the default stream), synchronised
 * before return. x and y are caller-owned device buffers of n doubles. */
int pb_selftest_exp(pb_ctx* ctx, const double* x, double* y, int64_t n, void* stream);
/* Arithmetic peak of this GPU by microbenchmark (the denominator of the pair
 * and near-field kernels' rooflines): independent fused multiply-add chains on
 * four CTAs of 256 threads per SM, the best of three timed launches of about
 * 20 ms. kind 0 = FP32 fma.rn.f32, 1 = FP64 fma.rn.f64, 2 = packed
 * fma.rn.f32x2 (two FMAs per instruction). *fma_per_s receives FMAs per second
 * (a flop count is twice that). Not in the paper. */
int pb_measure_peak(pb_ctx* ctx, int kind, double* fma_per_s);
/* Number of kernels this library has launched in this process (all kinds;
 * a kernel inside a replayed CUDA graph counts once per replay). */
int64_t pb_launch_count(void);
/* GMRES iterations (pb_solve, pb_solvation_energy, the request server) are
 * captured into a CUDA graph at their second iteration and replayed from then
 * on (1, the default; the environment variable PBBEM_GRAPHS=0 starts with 0),
 * or launched kernel by kernel (0). The same kernels run either way, so
 * results are bitwise the same. Applies to solves started after the call. */
int pb_set_graphs(pb_ctx* ctx, int enable);

/* ---- treecode far field ---------------------------------------------------- */
/* The paper computes its far field with a fast multipole method; this library
 * sums it directly by default. With the treecode enabled (1), FP32 operator
 * applications (the inner iterations of PB_MIXED solves, PB_F32 calls) of
 * meshes with at least min_points far-rule points use a kd-tree of the points
 * (leaves of 128): well-separated clusters (radius sum < theta x centre
 * distance) act through (order+1)^3 proxy sources on Chebyshev points of their
 * box, carrying the interpolated densities; all other pairs are summed
 * directly. The split-coordinate and FP64 applications (PB_MIXED's outer
 * residual, PB_F64 solves) stay direct, so mixed solves converge to the same
 * solution. order 2..7, theta in (0, 1]. Default: enabled, order 6, theta 0.7,
 * min_points 50000 (below that the direct sum is as fast on this GPU), or
 * disabled when the environment variable PBBEM_TREECODE=0 is set at pb_init.
 * The tree is built on the mesh's first
 * treecode application (host work and a device allocation; before any stream
 * capture). Applies to applications started after the call. */
int pb_set_treecode(pb_ctx* ctx, int enable, int order, double theta, int64_t min_points);
/* Sizes of a mesh's tree after its first treecode application: out[0..5] =
 * leaves, proxied clusters, far (proxy) list entries, near list entries,
 * direct point pairs and proxy point pairs of one application. */
int pb_tree_info(const pb_mesh* mesh, int64_t out[6]);

#ifdef __cplusplus
}
#endif
#endif /* PBBEM_H */
