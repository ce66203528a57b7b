// Internal declarations of the pbbem library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "pbbem.h"

namespace pb {

// ---------------------------------------------------------------- errors
int set_error(int code, const char* fmt, ...);
#define PB_CUDA(call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return ::pb::set_error(PB_ECUDA, "%s failed: %s (%s:%d)", #call,                 \
                                   cudaGetErrorString(e_), __FILE__, __LINE__);              \
    } while (0)
#define PB_TRY(expr)            \
    do {                        \
        int rc_ = (expr);       \
        if (rc_ != PB_OK) return rc_; \
    } while (0)

// ------------------------------------------------------- operator indices
// Operators stored by the near field, in this order (T is K transposed).
enum Op { O_M = 0, O_VL, O_KL, O_TL, O_DL, O_VY, O_KY, O_TY, O_DY, O_N };
// Near-field value arrays as stored (T is read through the transpose map).
enum NearVal { N_VL = 0, N_KL, N_DL, N_VY, N_KY, N_DY, N_M, N_VALS };

// A 2x2 block operator: block (r, c) = sum_o coef[r][c][o] * A_o, acting on
// x = [u; v] (c = 0: u, the Dirichlet trace; c = 1: v, the Neumann trace).
struct BlockOp {
    double c[2][2][O_N];
};

// Far-field work of one block operator, split into the two kernel row kinds:
//   phi-row: V (on v) and K (on u) terms, tested with lambda_a;
//   DT-row:  D (on u) and T (on v) terms (hypersingular and adjoint double layer).
struct FarPlan {
    int mode;          // 0: both rows phi-rows (VK2); 1: one phi-row + one DT-row (VKDT)
    int out_row[2];    // output block of kernel row 0 and row 1
    // kernel row 0 (phi-row): cVL, cVY, cKL, cKY
    // kernel row 1: phi-row (cVL, cVY, cKL, cKY) or DT-row (cDL, cDY, cTL, cTY)
    double k[2][4];
    double kappa;
    bool any;          // any far-field term at all
};

// The regular triangle rule, passed to kernels by value.
struct Rule {
    double l[6][3];
    double w[6];
    int Q;
};

// ------------------------------------------------------------- handles
struct Workspace {
    void* ptr = nullptr;
    size_t bytes = 0;
    // generation counter bumped when the buffer moves or is freed: its owning
    // mesh's (graphs capturing that mesh's work check it), or null for the
    // process-wide counter
    uint64_t* gen = nullptr;
};

}  // namespace pb

namespace pb {
struct KernelStats {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;  // unresolved launches
    int64_t launches = 0;
    double ms = 0.0, pairs = 0.0, ops = 0.0;
};
void count_launch(int n = 1);

// A launch sequence captured once into a CUDA graph and then replayed (the
// body of one GMRES iteration). Kernel launches and profiled pair-kernel
// launches seen while capturing are credited again on every replay.
struct CapturedTimer {
    int id;
    cudaEvent_t e0, e1;
    double pairs, ops;
    double pairs_j;  // + pairs_j x (j + 1) for the Arnoldi step j the replay runs
};
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    uint64_t gen = 0;                  // workspace generation the graph's pointers belong to
    int64_t launches = 0;              // kernels per replay
    int applies = 0;                   // operator applications per replay
    std::vector<CapturedTimer> timers;  // event pairs recorded by every replay
    bool failed = false;               // capture was refused: run the body directly
};
StepGraph* capturing();  // the graph this thread is capturing, or null
// Counts workspace (re)allocations: a captured graph whose generation differs
// may hold a freed pointer and must be captured again. The generation a graph
// depends on is the process-wide counter plus the counters of the meshes whose
// workspaces it uses (d0, d1; null: none), so that a mesh loaded or freed for
// one request does not invalidate the graphs of another.
uint64_t ws_generation(const uint64_t* d0 = nullptr, const uint64_t* d1 = nullptr);
void ws_bump();  // a buffer a graph may hold was freed (process-wide)
// Drop g if a workspace it depends on has moved since it was captured.
void graph_check(StepGraph& g, const uint64_t* d0 = nullptr, const uint64_t* d1 = nullptr);
// Capture body() on stream s (nothing runs); on failure g.failed is set and
// PB_OK returned so that the caller runs the body directly.
int graph_capture(StepGraph& g, cudaStream_t s, const std::function<int()>& body, const uint64_t* d0 = nullptr,
                  const uint64_t* d1 = nullptr);
int graph_replay(StepGraph& g, cudaStream_t s);
// after a replay has completed: its profiled launches into the context's
// statistics; j = the Arnoldi step the replay ran (work that grows with j)
int graph_credit(pb_ctx* ctx, StepGraph& g, int j = 0);
// the Arnoldi step the calling thread's GMRES is at (profiling of launches
// whose work grows with j; set by the GMRES loop before each iteration)
int& arnoldi_j();
void graph_free(StepGraph& g);
}  // namespace pb

namespace pb {
// Autotuned choice of the FP32 far-field launch for one size bucket
// (log2 of the point count) and row mode / precision.
struct TuneEntry {
    int kernel = 0;          // 0 = not tuned, 1 = scalar, 2 = packed f32x2
    double split_scale = 1;  // multiplier of the wave-filling split count
    int shape = 0;           // launch shape of the packed kernel (tile records, stages, targets per thread)
};
constexpr int TUNE_BUCKETS = 40;
struct PbTree;  // treecode of a mesh (tree.cu)
}  // namespace pb

struct pb_ctx {
    int profile = 0;
    int pair_kernel = 2;  // FP32 far-field kernel: 2 = packed f32x2 (default), 1 = scalar
    pb::TuneEntry tune[2][2][pb::TUNE_BUCKETS];  // [mode][accurate][bucket]
    pb::KernelStats stats[PB_KERNEL_COUNT];
    int device = 0;
    int num_sms = 0;
    int cc_major = 0, cc_minor = 0;
    void* encode_tiled = nullptr;  // cuTensorMapEncodeTiled entry point
    int graphs = 1;                // replay GMRES iterations from CUDA graphs
    // treecode far field for FP32 applications (inner iterations)
    int tree_enable = 1;           // on by default for meshes of at least tree_min_points points
    int tree_order = 6;            // Chebyshev points per dimension - 1
    double tree_theta = 0.7;       // separation: radius sum < theta x centre distance
    int64_t tree_min_points = 50000;
};

struct pb_mesh {
    pb_ctx* ctx = nullptr;
    int64_t nv = 0, nt = 0, np = 0;
    int Q = 0, n_ss = 0;
    double ctr[3] = {0.0, 0.0, 0.0};  // centre of the bounding box: origin of the split FP32 coordinates
    int n_ss_cls[3] = {0, 0, 0};  // singular Gauss points per dimension: coincident, edge, vertex pairs
    double rule_l[6][3];
    double rule_w[6];
    // distance band of the plan, and its reference rule (right-hand side and
    // energy): the band rule with a band, the far rule without
    double band_eta = 0.0;
    int Qr = 0;
    int64_t np_ref = 0;
    double ref_l[6][3];
    double ref_w[6];
    // device arrays
    double* verts = nullptr;    // nv x 3
    int32_t* tris = nullptr;    // nt x 3
    double* tgeo = nullptr;     // nt x 16: n(3), area, e0(3), e1(3), e2(3), pad(3)
    double* pts64 = nullptr;    // np x 4: x, y, z, w (rule weight x area)
    double* pts_ref = nullptr;  // np_ref x 4: points of the reference rule (== pts64 without a band)
    float* pts32 = nullptr;     // np x 4: x, y, z, w rounded to float
    float* pts32lo = nullptr;   // np x 4: x - float(x), ..., 0
    int32_t* v2t_ptr = nullptr; // nv + 1
    int32_t* v2t = nullptr;     // 3 nt entries: tri * 3 + local vertex
    // adjacent triangle pairs (share a vertex), ordered by (ti, tj)
    int64_t npairs = 0, n_adj = 0;  // npairs = n_adj + n_band
    int4* pairs = nullptr;      // n_adj: (ti, tj, kind, perms): kind 0 coincident, 1 edge, 2 vertex
    int32_t* adj_ptr = nullptr;    // nt + 1: pairs of triangle t
    int32_t* pair_rev = nullptr;   // index of the reversed pair (tj, ti)
    int32_t* pair_coin = nullptr;  // coincident pairs
    int32_t* pair_prim = nullptr;  // adjacent pairs with ti < tj (each also gives its reverse)
    int64_t n_coin = 0, n_prim = 0, n_prim_edge = 0;  // (the rest of n_prim share one vertex)
    // band pairs (no shared vertex, within the plan's band), ordered by (ti, tj):
    // band pair q is (band_t[q], band_s[q]); triangle t's are band_ptr[t]..band_ptr[t+1]
    int64_t n_band = 0;
    int32_t* band_ptr = nullptr;
    int32_t* band_s = nullptr;
    int32_t* band_t = nullptr;
    // vertex-pair pattern of the near field (symmetric)
    int64_t nnz = 0;
    int max_row = 0;            // longest row of the pattern
    int32_t* row_ptr = nullptr; // nv + 1
    int32_t* col = nullptr;     // nnz
    int32_t* tpos = nullptr;    // nnz: index of the transposed entry
    int32_t* row_of = nullptr;  // nnz: row of each entry
    int32_t* diag_pos = nullptr;// nv
    int* status = nullptr;          // device status word of bounded waits (0 = fine)
    // workspaces (grown on demand)
    pb::Workspace ws_src, ws_part, ws_tri, ws_vec, ws_comb, ws_tree;
    uint64_t ws_gen = 0;  // bumped when one of the workspaces above moves or is freed
    pb::PbTree* tree = nullptr;  // built on the first treecode application
    size_t device_bytes = 0;
};

struct pb_near {
    const pb_mesh* mesh = nullptr;
    double kappa = 0.0;
    double* val = nullptr;   // N_VALS x nnz (near part = regularised - far rule; M exact)
    double* diag = nullptr;  // N_VALS x nv: full operator diagonals
    // the mass matrix alone on its own pattern (vertices sharing a triangle)
    int32_t* mrow_ptr = nullptr;  // nv + 1
    int32_t* mcol = nullptr;
    double* mval = nullptr;
};

namespace pb {

inline Rule mesh_rule(const pb_mesh* m) {
    Rule r;
    for (int q = 0; q < 6; ++q) {
        for (int c = 0; c < 3; ++c) r.l[q][c] = m->rule_l[q][c];
        r.w[q] = m->rule_w[q];
    }
    r.Q = m->Q;
    return r;
}
// the plan's reference rule (band rule with a band, else the far rule)
inline Rule mesh_ref_rule(const pb_mesh* m) {
    Rule r;
    for (int q = 0; q < 6; ++q) {
        for (int c = 0; c < 3; ++c) r.l[q][c] = m->ref_l[q][c];
        r.w[q] = m->ref_w[q];
    }
    r.Q = m->Qr;
    return r;
}

// exclusive scan of n counts into ptr[0..n] on stream s; *total (device) = the sum
int device_scan(int64_t n, const int32_t* cnt, int32_t* ptr, int64_t* total, cudaStream_t s);

// device allocation helpers (track bytes on the mesh)
int dev_alloc(void** p, size_t bytes);
int ws_reserve(Workspace& w, size_t bytes);
void ws_free(Workspace& w);

// formulation -> block operators (system, Calderon operators, RHS scaling)
int system_blockop(const pb_params* prm, int form, double alpha, double beta, BlockOp* out);
int calderon_blockop(const pb_params* prm, int form, int which /*0 int, 1 ext*/, BlockOp* out);
bool form_is_exterior(int form);
int make_far_plan(const BlockOp& B, double kappa, FarPlan* out);

// a3 + a4 + a5: y = B x (x, y device, 2 nv doubles). comb: B's near values
// already combined (4 nnz doubles then 4 nnz floats, from combine_near), or
// null to combine them into the mesh's workspace first.
int apply_blockop(const pb_mesh* m, const pb_near* nf, const BlockOp& B, int prec, const double* x,
                  double* y, cudaStream_t s, const double* comb = nullptr);
// near values combined for a block operator (FP64 and FP32 copies) and diagonals
int combine_near(const pb_mesh* m, const pb_near* nf, const BlockOp& B, double* comb64, float* comb32,
                 cudaStream_t s);

// batched application over several meshes (one pair-kernel launch per row mode)
struct FarJob {
    const pb_mesh* m;
    const pb_near* nf;
    BlockOp B;
    const double* x;
    double* y;
    cudaStream_t s = nullptr;  // the job's own stream for its per-job kernels (null: the batch's stream)
    const double* comb = nullptr;  // B's combined near values (null: combined into the mesh's workspace)
};
struct BatchScratch {
    BatchScratch() { table.gen = &table_gen; }
    uint64_t table_gen = 0;           // the table's own counter: no captured graph uses the table
    Workspace table;                  // job and work-item tables on the device
    std::vector<cudaEvent_t> ev;      // per job: its stream's work before the shared launch
    cudaEvent_t ev_main = nullptr;    // the shared launch, before the jobs' own reductions
};
void batch_scratch_free(BatchScratch& bs);
int apply_blockops_batched(const std::vector<FarJob>& jobs, int prec, BatchScratch& bs, cudaStream_t s);

// treecode far field (FP32): per-target partial sums in the direct kernel's
// split layout, in the mesh's ws_part (*part_out, *nsplit slices); the tree is
// built on first use
int tree_far(const pb_mesh* m, const FarPlan& fp, const double* x, bool need_u, bool need_v, float** part_out,
             int* nsplit, cudaStream_t s);
void tree_free(PbTree* t);
int tree_info(const pb_mesh* m, int64_t out[6]);

// far-field split count for the pair kernels
int far_splits(const pb_mesh* m, int targets_per_cta, int ctas_per_sm);
// largest split count the packed kernels use for np points (workspace estimates)
int far_splits_estimate(pb_ctx* ctx, int64_t np);
// the tuned entry that applies to np points (kernel 0 when none)
TuneEntry tuned(const pb_ctx* ctx, int64_t np, int mode, bool acc);
int tune_bucket(int64_t np);

// Chebyshev solve with the mass matrix: y = M^-1 x on both halves of a 2 nv vector
int mass_solve(const pb_mesh* m, const pb_near* nf, const double* x, double* y, double* work,
               int iters, cudaStream_t s);

// CUDA events around one launch on its stream, when the context profiles.
// Host worker pool, created on first use and kept for the life of the process:
// host_parallel(n, f) calls f(0) ... f(n - 1) across the workers and the
// calling thread and returns when all have returned. A call made while
// another is running (another host thread) runs its jobs on the caller alone.
int host_threads();
void host_parallel(int n, const std::function<void(int)>& f);

// Host-side phase trace: with PBBEM_TRACE set in the environment, lap() prints
// the wall time since the previous lap (stderr), after synchronising the device
// so that the time belongs to the phase that queued the work.
struct PhaseTrace {
    const char* scope;
    double t0;
    bool on;
    explicit PhaseTrace(const char* s);
    void lap(const char* label);
    void note(const char* label, double value) const;  // a value beside the laps (no timing)
};

struct Timer {
    pb_ctx* ctx;
    int id;
    cudaStream_t s;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double pairs, ops;
    double pairs_j;  // work that grows with the Arnoldi step: pairs + pairs_j (j + 1)
    Timer(pb_ctx* c, int k, cudaStream_t st, double p, double o, double pj = 0.0)
        : ctx(c), id(k), s(st), pairs(p), ops(o), pairs_j(pj) {
        if (ctx && ctx->profile && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess)
            record(e0);
    }
    // inside a stream capture an event record becomes a graph node only when
    // marked external (otherwise it only orders the captured work)
    void record(cudaEvent_t e) {
        if (capturing()) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
        else cudaEventRecord(e, s);
    }
    void stop() {
        if (!e1) return;
        record(e1);
        if (StepGraph* g = capturing()) {  // recorded again by every replay
            g->timers.push_back({id, e0, e1, pairs, ops, pairs_j});
            e0 = e1 = nullptr;
            return;
        }
        KernelStats& st = ctx->stats[id];
        const double p = pairs + pairs_j * (double)(arnoldi_j() + 1);
        st.events.push_back({e0, e1});
        st.launches += 1;
        st.pairs += p;
        st.ops += p * ops;
        e0 = e1 = nullptr;
    }
};

}  // namespace pb
