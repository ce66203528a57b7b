// a1: mesh ingest - validation, topology, quadrature points, adjacent
// triangle pairs and the vertex-pair pattern of the near field.
//
// Paper, "Numerical discretization": continuous piecewise-linear Galerkin
// elements on a triangular surface mesh, one unknown per vertex. Far
// (non-adjacent) triangle pairs are integrated with one symmetric triangle
// rule on both triangles; pairs that share a vertex are singular and get the
// regularised rule of the near field (near.cu). With a distance band in the
// quadrature plan, non-adjacent pairs closer than band_eta times the sum of
// their radii are listed too: the near field adds to them the difference of
// the finer band rule and the far rule.
//
// The host work (adjacent pairs, near pattern) runs on several threads; every
// list is built per triangle or per vertex row, so its order does not depend
// on the thread count. The band search runs on the device.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

#include "internal.h"

namespace pb {

// Symmetric triangle rules in barycentric coordinates, weights summing to 1.
// 6 points, degree 4 (Dunavant 1985: two orbits of 3); 3 points, degree 2;
// 1 point (centroid).
static void rule_points(int q, double l[6][3], double w[6]) {
    if (q == 6) {
        const double a[2] = {0.445948490915965, 0.091576213509771};
        const double wt[2] = {0.223381589678011, 0.109951743655322};
        for (int o = 0; o < 2; ++o)
            for (int k = 0; k < 3; ++k) {
                for (int c = 0; c < 3; ++c) l[3 * o + k][c] = a[o];
                l[3 * o + k][k] = 1.0 - 2.0 * a[o];
                w[3 * o + k] = wt[o];
            }
    } else if (q == 3) {
        for (int k = 0; k < 3; ++k) {
            for (int c = 0; c < 3; ++c) l[k][c] = 1.0 / 6.0;
            l[k][k] = 2.0 / 3.0;
            w[k] = 1.0 / 3.0;
        }
    } else {
        for (int c = 0; c < 3; ++c) l[0][c] = 1.0 / 3.0;
        w[0] = 1.0;
    }
}


// Per-triangle geometry and the quadrature points (FP64, plus float copies
// relative to the mesh centre split into hi and lo parts).
__global__ void k_geometry(const double* __restrict__ verts, const int32_t* __restrict__ tris,
                           int64_t nt, Rule rule, Rule ref, double cx, double cy, double cz,
                           double* __restrict__ tgeo, double* __restrict__ pts64,
                           float* __restrict__ pts32, float* __restrict__ pts32lo, double* __restrict__ pts_ref) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double p[3][3];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) p[a][k] = verts[3 * (int64_t)tris[3 * t + a] + k];
    double u[3], v[3], n[3];
    for (int k = 0; k < 3; ++k) {
        u[k] = p[1][k] - p[0][k];
        v[k] = p[2][k] - p[0][k];
    }
    n[0] = u[1] * v[2] - u[2] * v[1];
    n[1] = u[2] * v[0] - u[0] * v[2];
    n[2] = u[0] * v[1] - u[1] * v[0];
    double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double area = 0.5 * len;
    double* g = tgeo + 16 * t;
    for (int k = 0; k < 3; ++k) g[k] = n[k] / len;
    g[3] = area;
    for (int k = 0; k < 3; ++k) {
        g[4 + k] = p[2][k] - p[1][k];   // edge opposite vertex 0
        g[7 + k] = p[0][k] - p[2][k];   // opposite vertex 1
        g[10 + k] = p[1][k] - p[0][k];  // opposite vertex 2
    }
    g[13] = g[14] = g[15] = 0.0;
    const double c[3] = {cx, cy, cz};
    for (int q = 0; q < rule.Q; ++q) {
        int64_t i = t * rule.Q + q;
        double x[3];
        for (int k = 0; k < 3; ++k)
            x[k] = rule.l[q][0] * p[0][k] + rule.l[q][1] * p[1][k] + rule.l[q][2] * p[2][k];
        double w = rule.w[q] * area;
        for (int k = 0; k < 3; ++k) {
            pts64[4 * i + k] = x[k];
            double rel = x[k] - c[k];
            float hi = (float)rel;
            pts32[4 * i + k] = hi;
            pts32lo[4 * i + k] = (float)(rel - (double)hi);
        }
        pts64[4 * i + 3] = w;
        pts32[4 * i + 3] = (float)w;
        pts32lo[4 * i + 3] = 0.0f;
    }
    if (pts_ref)  // the plan's reference rule (right-hand side and energy), when it differs
        for (int q = 0; q < ref.Q; ++q) {
            int64_t i = t * ref.Q + q;
            for (int k = 0; k < 3; ++k)
                pts_ref[4 * i + k] = ref.l[q][0] * p[0][k] + ref.l[q][1] * p[1][k] + ref.l[q][2] * p[2][k];
            pts_ref[4 * i + 3] = ref.w[q] * area;
        }
}

// ---- distance band on the device. The test uses the same IEEE operations,
// in the same order and without contraction, as the host code that computed
// the centroids and radii (and as the oracle), so every decision is the same.
__device__ __forceinline__ bool band_hit(const double* __restrict__ C, const double* __restrict__ R, int64_t t,
                                         int64_t s, double eta) {
    const double d0 = __dsub_rn(C[3 * t], C[3 * s]), d1 = __dsub_rn(C[3 * t + 1], C[3 * s + 1]),
                 d2 = __dsub_rn(C[3 * t + 2], C[3 * s + 2]);
    const double q = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
    const double lim = __dmul_rn(eta, __dadd_rn(R[t], R[s]));
    return q < __dmul_rn(lim, lim);
}

__device__ __forceinline__ bool share_vertex_dev(const int32_t* a, const int32_t* b) {
    bool r = false;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) r |= a[i] == b[j];
    return r;
}

struct BandGrid {
    const double* C;      // nt x 3 centroids
    const double* R;      // nt radii
    const float4* CR32;   // nt: centroid relative to the box centre, radius, in FP32 (the prefilter)
    float slack;          // absolute margin of the prefilter: 4 x 2^-23 x the largest centred coordinate
    const int32_t* cstart;  // ncell + 1
    const int32_t* ctri;    // triangles by cell
    const int32_t* tcell;   // cell of each triangle
    int64_t dim[3];
    double eta;
};

// FP32 prefilter of the band test: true only where the FP64 test (band_hit)
// is certain to fail. Rounding the centred coordinates to FP32 moves each
// centroid difference by at most 2 x 2^-24 x the largest centred coordinate,
// and the FP32 operations change the distance and the limit by a few units of
// 2^-24 relative; the test demands a distance above 1.001 limits plus more
// than twice that absolute error (the slack), far outside either.
__device__ __forceinline__ bool band_far32(const float4& a, const float4& b, float eta, float slack) {
    const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z;
    const float q = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
    const float lim = fmaf(1.001f * eta, a.w + b.w, slack);
    return q > lim * lim;
}

// One warp per triangle, lanes over the candidates of the 27 cells around its
// cell. Pass 0 counts the band partners of each triangle; pass 1 writes them
// (sorted) with their owner: the hits are compacted in candidate order into
// the owner slots (scratch), then each one is placed at its rank among them
// (the partners are distinct), and the owner slots are filled.
__global__ void k_band_search(int64_t nt, const int32_t* __restrict__ tris, BandGrid g, int pass,
                              int32_t* __restrict__ cnt, const int32_t* __restrict__ ptr, int32_t* __restrict__ bs,
                              int32_t* __restrict__ bt) {
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= nt) return;  // whole warps
    const int64_t c = g.tcell[t];
    const int64_t c0 = c % g.dim[0], c1 = (c / g.dim[0]) % g.dim[1], c2 = c / (g.dim[0] * g.dim[1]);
    const int32_t* ft = tris + 3 * t;
    const float4 ct = g.CR32[t];
    const float eta32 = (float)g.eta;
    int n = 0;  // hits so far (the same in every lane)
    const int64_t base = pass ? ptr[t] : 0;
    for (int64_t z = max((int64_t)0, c2 - 1); z <= min(g.dim[2] - 1, c2 + 1); ++z)
        for (int64_t y = max((int64_t)0, c1 - 1); y <= min(g.dim[1] - 1, c1 + 1); ++y)
            for (int64_t x = max((int64_t)0, c0 - 1); x <= min(g.dim[0] - 1, c0 + 1); ++x) {
                const int64_t cc = x + g.dim[0] * (y + g.dim[1] * z);
                const int32_t k1 = g.cstart[cc + 1];
                for (int32_t kb = g.cstart[cc]; kb < k1; kb += 32) {
                    const int32_t k = kb + lane;
                    int32_t s = 0;
                    bool hit = false;
                    if (k < k1) {
                        s = g.ctri[k];
                        hit = s != (int32_t)t && !band_far32(ct, g.CR32[s], eta32, g.slack) &&
                              band_hit(g.C, g.R, t, s, g.eta) && !share_vertex_dev(ft, tris + 3 * (int64_t)s);
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, hit);
                    if (pass && hit) bt[base + n + __popc(m & ((1u << lane) - 1u))] = s;
                    n += __popc(m);
                }
            }
    if (!pass) {
        if (lane == 0) cnt[t] = n;
        return;
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
        const int32_t v = bt[base + i];
        int r = 0;
        for (int j = 0; j < n; ++j) r += bt[base + j] < v;
        bs[base + r] = v;
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) bt[base + i] = (int32_t)t;
}

// exclusive scan of n counts into ptr[0..n] (one block; n up to 2^28), total in ptr[n]
__global__ void k_scan(int64_t n, const int32_t* __restrict__ cnt, int32_t* __restrict__ ptr,
                       int64_t* __restrict__ total) {
    __shared__ int64_t part[1024];
    const int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = threadIdx.x * chunk, b1 = min(n, b0 + chunk);
    int64_t s = 0;
    for (int64_t i = b0; i < b1; ++i) s += cnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            const int64_t v = part[k];
            part[k] = acc;
            acc += v;
        }
        *total = acc;
        ptr[n] = (int32_t)min(acc, (int64_t)INT32_MAX);
    }
    __syncthreads();
    int64_t acc = part[threadIdx.x];
    for (int64_t i = b0; i < b1; ++i) {
        ptr[i] = (int32_t)min(acc, (int64_t)INT32_MAX);
        acc += cnt[i];
    }
}

// ---- near pattern on the device: row i holds every vertex of every triangle
// paired (adjacent or band) with a triangle at i. One warp per row inserts the
// candidates into a shared-memory hash set of PAT_HASH slots (a power of two),
// compacts it, and (pass 1) writes the columns in increasing order (each one's
// rank among the row's values). The candidates repeat each column many times
// (every triangle pair that reaches it), so pass 0 starts from a small set and
// reports in *ovf a row that did not fit (the host then retries with a larger
// set, up to twice the largest candidate count); pass 1 is sized from the
// largest column count that pass 0 found.

// candidates of each row (with repetitions): an upper bound of its columns
__global__ void k_row_candidates(int64_t nv, const int32_t* __restrict__ v2t_ptr, const int32_t* __restrict__ v2t,
                                 const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ band_ptr,
                                 int* __restrict__ maxc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nv) return;
    int64_t c = 0;
    for (int32_t k = v2t_ptr[i]; k < v2t_ptr[i + 1]; ++k) {
        const int32_t t = v2t[k] / 3;
        c += 3 * (int64_t)(adj_ptr[t + 1] - adj_ptr[t]);
        if (band_ptr) c += 3 * (int64_t)(band_ptr[t + 1] - band_ptr[t]);
    }
    atomicMax(maxc, (int)min(c, (int64_t)INT32_MAX));
}

__global__ void k_row_pattern(int64_t nv, int pass, int PAT_HASH, int PAT_WARPS, const int32_t* __restrict__ v2t_ptr,
                              const int32_t* __restrict__ v2t, const int32_t* __restrict__ tris,
                              const int32_t* __restrict__ adj_ptr, const int4* __restrict__ pairs,
                              const int32_t* __restrict__ band_ptr, const int32_t* __restrict__ band_s,
                              int32_t* __restrict__ cnt, int* __restrict__ maxrow, const int32_t* __restrict__ row_ptr,
                              int32_t* __restrict__ col, int* __restrict__ ovf, int* __restrict__ status) {
    extern __shared__ int32_t psm[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * PAT_WARPS + w;
    if (i >= nv) return;  // whole warps
    int32_t* tb = psm + (size_t)w * (PAT_HASH + PAT_HASH / 2);
    int32_t* ls = tb + PAT_HASH;
    for (int k = lane; k < PAT_HASH; k += 32) tb[k] = -1;
    __syncwarp();
    bool full = false;
    for (int32_t k = v2t_ptr[i]; k < v2t_ptr[i + 1]; ++k) {
        const int32_t t = v2t[k] / 3;
        const int32_t p0 = adj_ptr[t], L1 = adj_ptr[t + 1] - p0;
        const int32_t q0 = band_ptr ? band_ptr[t] : 0, L2 = band_ptr ? band_ptr[t + 1] - q0 : 0;
        const int total = 3 * (L1 + L2);
        for (int c = lane; c < total; c += 32) {
            const int idx = c / 3, b = c - 3 * idx;
            const int32_t sidx = idx < L1 ? pairs[p0 + idx].y : band_s[q0 + idx - L1];
            const int32_t j = tris[3 * (int64_t)sidx + b];
            uint32_t h = ((uint32_t)j * 2654435761u) & (PAT_HASH - 1);
            int probe = 0;
            for (; probe < PAT_HASH; ++probe) {
                const int32_t old = atomicCAS(&tb[h], -1, j);
                if (old == -1 || old == j) break;
                h = (h + 1) & (PAT_HASH - 1);
            }
            full |= probe == PAT_HASH;
        }
        if (__any_sync(0xffffffffu, full)) break;  // the set is too small for this row
    }
    __syncwarp();
    int n = 0;
    for (int base = 0; base < PAT_HASH; base += 32) {
        const int32_t v = tb[base + lane];
        const unsigned bal = __ballot_sync(0xffffffffu, v >= 0);
        if (v >= 0) {
            const int pos = n + __popc(bal & ((1u << lane) - 1));
            if (pos < PAT_HASH / 2) ls[pos] = v;
        }
        n += __popc(bal);
    }
    full = __any_sync(0xffffffffu, full) || n > PAT_HASH / 2;
    if (full) {
        if (lane == 0) atomicExch(pass == 0 ? ovf : status, PB_EINVAL);
        return;
    }
    if (pass == 0) {
        if (lane == 0) {
            cnt[i] = n;
            atomicMax(maxrow, n);
        }
        return;
    }
    __syncwarp();
    const int32_t r0 = row_ptr[i];
    for (int k = lane; k < n; k += 32) {
        const int32_t v = ls[k];
        int rank = 0;
        for (int q = 0; q < n; ++q) rank += ls[q] < v;
        col[r0 + rank] = v;
    }
}

int device_scan(int64_t n, const int32_t* cnt, int32_t* ptr, int64_t* total, cudaStream_t s) {
    k_scan<<<1, 1024, 0, s>>>(n, cnt, ptr, total);
    ::pb::count_launch();
    PB_CUDA(cudaGetLastError());
    return PB_OK;
}

// transposed positions, diagonal positions and the row of every nonzero
// one warp per row i, lanes over its entries: the position of each entry's
// transpose, the row of each entry and the diagonal's position
__global__ void k_pattern_maps(int64_t nv, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                               int32_t* __restrict__ tpos, int32_t* __restrict__ diag_pos, int32_t* __restrict__ row_of,
                               int* __restrict__ status) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= nv) return;
    for (int32_t k = row_ptr[i] + lane; k < row_ptr[i + 1]; k += 32) {
        const int32_t j = col[k];
        row_of[k] = (int32_t)i;
        int32_t lo = row_ptr[j], hi = row_ptr[j + 1];
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (col[mid] < (int32_t)i) lo = mid + 1;
            else hi = mid;
        }
        if (lo >= row_ptr[j + 1] || col[lo] != (int32_t)i) {
            atomicExch(status, PB_EMESH);
            continue;
        }
        tpos[k] = lo;
        if (j == (int32_t)i) diag_pos[i] = k;
    }
}

constexpr int MAX_HOST_THREADS = 16;

// f(chunk, begin, end) over [0, n) in contiguous chunks on the host worker
// pool; returns the number of chunks (chunk c covers [n c / k, n (c + 1) / k))
template <class F>
static int parallel_chunks(int64_t n, F&& f) {
    const int nth = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::min(host_threads(), MAX_HOST_THREADS), (n + 2047) / 2048));
    host_parallel(nth, [&](int i) { f(i, n * i / nth, n * (i + 1) / nth); });
    return nth;
}

static int upload(void** dst, const void* src, size_t bytes, size_t* total) {
    PB_TRY(dev_alloc(dst, bytes));
    if (bytes) PB_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    *total += bytes;
    return PB_OK;
}

static void free_mesh_arrays(pb_mesh* m) {
    PhaseTrace tr("mesh_free");
    void* ptrs[] = {m->verts,    m->tris,     m->tgeo,     m->pts64,   m->pts32,  m->pts32lo, m->v2t_ptr,
                    m->v2t,      m->pairs,    m->adj_ptr,  m->row_ptr, m->col,    m->tpos,    m->row_of,
                    m->diag_pos, m->status,   m->pair_rev, m->pair_coin, m->pair_prim, m->band_ptr, m->band_s,
                    m->band_t};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (m->pts_ref && m->pts_ref != m->pts64) cudaFree(m->pts_ref);
    ws_free(m->ws_src);
    ws_free(m->ws_part);
    ws_free(m->ws_tri);
    ws_free(m->ws_vec);
    ws_free(m->ws_comb);
    ws_free(m->ws_tree);
    tree_free(m->tree);
    m->tree = nullptr;
    tr.lap("all");
}

static int load(pb_ctx* ctx, const double* verts_in, int64_t nv, const int32_t* tris_in, int64_t nt,
                const pb_quad_plan* plan, int mem, pb_mesh* m) {
    if (nv < 4 || nt < 4) return set_error(PB_EMESH, "mesh too small (%lld verts, %lld tris)",
                                           (long long)nv, (long long)nt);
    if (nt > (int64_t)1 << 28 || nv > (int64_t)1 << 28)
        return set_error(PB_EINVAL, "mesh too large for 32-bit indices");
    int Q = plan ? plan->far_q : 6;
    int nss = plan ? plan->n_ss : 4;
    const double eta = plan ? plan->band_eta : 0.0;
    const int bq = plan && plan->band_q ? plan->band_q : 6;
    if (Q != 1 && Q != 3 && Q != 6) return set_error(PB_EINVAL, "far_q must be 1, 3 or 6 (got %d)", Q);
    if (nss < 1 || nss > 12) return set_error(PB_EINVAL, "n_ss must be in 1..12 (got %d)", nss);
    int ncls[3] = {plan ? plan->n_ss_coin : 0, plan ? plan->n_ss_edge : 0, plan ? plan->n_ss_vert : 0};
    for (int c = 0; c < 3; ++c) {
        if (ncls[c] == 0) ncls[c] = nss;
        if (ncls[c] < 1 || ncls[c] > 12)
            return set_error(PB_EINVAL, "per-class singular orders must be 0 or in 1..12 (got %d)", ncls[c]);
    }
    if (!(eta >= 0.0) || !(eta <= 64.0)) return set_error(PB_EINVAL, "band_eta must be in [0, 64] (got %g)", eta);
    if (eta > 0.0 && ((bq != 3 && bq != 6) || bq <= Q))
        return set_error(PB_EINVAL, "band_q must be 3 or 6 and finer than far_q (got %d, far_q %d)", bq, Q);
    m->ctx = ctx;
    m->nv = nv;
    m->nt = nt;
    m->Q = Q;
    m->n_ss = nss;
    for (int c = 0; c < 3; ++c) m->n_ss_cls[c] = ncls[c];
    m->np = nt * Q;
    m->band_eta = eta;
    m->Qr = eta > 0.0 ? bq : Q;
    rule_points(Q, m->rule_l, m->rule_w);
    rule_points(m->Qr, m->ref_l, m->ref_w);

    PhaseTrace tr("mesh_load");
    std::vector<double> V(3 * nv);
    std::vector<int32_t> T(3 * nt);
    if (mem == PB_MEM_DEVICE) {
        PB_CUDA(cudaMemcpy(V.data(), verts_in, sizeof(double) * 3 * nv, cudaMemcpyDeviceToHost));
        PB_CUDA(cudaMemcpy(T.data(), tris_in, sizeof(int32_t) * 3 * nt, cudaMemcpyDeviceToHost));
    } else if (mem == PB_MEM_HOST) {
        memcpy(V.data(), verts_in, sizeof(double) * 3 * nv);
        memcpy(T.data(), tris_in, sizeof(int32_t) * 3 * nt);
    } else {
        return set_error(PB_EINVAL, "mem must be PB_MEM_HOST or PB_MEM_DEVICE");
    }

    tr.lap("copy_in");
    // ---- validation
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < nv; ++i)
        for (int k = 0; k < 3; ++k) {
            double x = V[3 * i + k];
            if (!std::isfinite(x)) return set_error(PB_EMESH, "vertex %lld is not finite", (long long)i);
            lo[k] = std::min(lo[k], x);
            hi[k] = std::max(hi[k], x);
        }
    double diag2 = 0.0;
    for (int k = 0; k < 3; ++k) diag2 += (hi[k] - lo[k]) * (hi[k] - lo[k]);
    double vol6 = 0.0;
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t* f = &T[3 * t];
        for (int a = 0; a < 3; ++a)
            if (f[a] < 0 || f[a] >= nv)
                return set_error(PB_EMESH, "triangle %lld has vertex index %d out of range", (long long)t, f[a]);
        if (f[0] == f[1] || f[1] == f[2] || f[0] == f[2])
            return set_error(PB_EMESH, "triangle %lld repeats a vertex", (long long)t);
        const double *p0 = &V[3 * f[0]], *p1 = &V[3 * f[1]], *p2 = &V[3 * f[2]];
        double u[3], w[3];
        for (int k = 0; k < 3; ++k) {
            u[k] = p1[k] - p0[k];
            w[k] = p2[k] - p0[k];
        }
        double c0 = u[1] * w[2] - u[2] * w[1], c1 = u[2] * w[0] - u[0] * w[2], c2 = u[0] * w[1] - u[1] * w[0];
        double a2 = c0 * c0 + c1 * c1 + c2 * c2;
        if (!(a2 > 1e-24 * diag2 * diag2))
            return set_error(PB_EMESH, "triangle %lld has (near) zero area", (long long)t);
        vol6 += p0[0] * (p1[1] * p2[2] - p1[2] * p2[1]) - p0[1] * (p1[0] * p2[2] - p1[2] * p2[0]) +
                p0[2] * (p1[0] * p2[1] - p1[1] * p2[0]);
    }
    tr.lap("validate");

    // ---- vertex -> triangle map
    std::vector<int32_t> v2t_ptr(nv + 1, 0), v2t(3 * nt);
    for (int64_t k = 0; k < 3 * nt; ++k) v2t_ptr[T[k] + 1]++;
    for (int64_t i = 0; i < nv; ++i) v2t_ptr[i + 1] += v2t_ptr[i];
    {
        std::vector<int32_t> fill(v2t_ptr.begin(), v2t_ptr.end() - 1);
        for (int64_t t = 0; t < nt; ++t)
            for (int a = 0; a < 3; ++a) v2t[fill[T[3 * t + a]]++] = (int32_t)(3 * t + a);
    }
    // every undirected edge must lie in exactly two triangles, traversed in
    // opposite directions: for the edge i -> j of triangle t, the triangles of
    // vertex i that follow i by j (t itself) and those that precede i by j
    {
        std::atomic<int64_t> first_bad{INT64_MAX};  // lowest failing 3 t + a (deterministic report)
        auto census = [&](int64_t t, int a, int* same, int* opp) {
            const int32_t i = T[3 * t + a], j = T[3 * t + (a + 1) % 3];
            *same = *opp = 0;
            for (int32_t k = v2t_ptr[i]; k < v2t_ptr[i + 1]; ++k) {
                const int64_t u = v2t[k] / 3;
                const int c = v2t[k] % 3;
                *same += T[3 * u + (c + 1) % 3] == j;
                *opp += T[3 * u + (c + 2) % 3] == j;
            }
        };
        parallel_chunks(nt, [&](int, int64_t b0, int64_t b1) {
            for (int64_t t = b0; t < b1; ++t)
                for (int a = 0; a < 3; ++a) {
                    int same, opp;
                    census(t, a, &same, &opp);
                    if (same != 1 || opp != 1) {
                        int64_t cur = first_bad.load();
                        while (3 * t + a < cur && !first_bad.compare_exchange_weak(cur, 3 * t + a)) {
                        }
                        return;
                    }
                }
        });
        const int64_t bad = first_bad.load();
        if (bad != INT64_MAX) {
            const int64_t t = bad / 3;
            const int a = (int)(bad % 3);
            int same, opp;
            census(t, a, &same, &opp);
            const int32_t i = T[3 * t + a], j = T[3 * t + (a + 1) % 3];
            const unsigned long long e0 = (unsigned long long)std::min(i, j), e1 = (unsigned long long)std::max(i, j);
            if (same + opp != 2)
                return set_error(PB_EMESH, "edge (%llu,%llu) is shared by %d triangles (mesh not closed or not "
                                 "manifold)", e0, e1, same + opp);
            return set_error(PB_EMESH, "edge (%llu,%llu) has the same direction in both triangles (inconsistent "
                             "orientation)", e0, e1);
        }
    }
    tr.lap("edges");
    if (!(vol6 > 0.0))
        return set_error(PB_EMESH, "enclosed volume is not positive (triangles must be counter-clockwise "
                         "seen from outside)");
    for (int64_t i = 0; i < nv; ++i)
        if (v2t_ptr[i + 1] == v2t_ptr[i])
            return set_error(PB_EMESH, "vertex %lld belongs to no triangle", (long long)i);

    tr.lap("v2t");
    // ---- adjacent triangle pairs (share >= 1 vertex), ordered by (ti, tj),
    // listed per triangle
    std::vector<int32_t> adj_ptr(nt + 1, 0);
    auto neighbours = [&](int64_t t, std::vector<int32_t>& mark, std::vector<int32_t>& nb) {
        nb.clear();
        for (int a = 0; a < 3; ++a) {
            int32_t i = T[3 * t + a];
            for (int32_t k = v2t_ptr[i]; k < v2t_ptr[i + 1]; ++k) {
                int32_t s = v2t[k] / 3;
                if (mark[s] != (int32_t)t) {
                    mark[s] = (int32_t)t;
                    nb.push_back(s);
                }
            }
        }
        std::sort(nb.begin(), nb.end());
    };
    // one pass: each chunk of triangles lists its pairs in its own buffer, in
    // triangle order; the buffers are then laid end to end
    std::vector<std::vector<int4>> chunk_pairs(MAX_HOST_THREADS);
    const int nchunk = parallel_chunks(nt, [&](int c, int64_t b0, int64_t b1) {
        std::vector<int32_t> mark(nt, -1), nb;
        std::vector<int4>& out = chunk_pairs[c];
        out.reserve((size_t)(b1 - b0) * 16);
        for (int64_t t = b0; t < b1; ++t) {
            neighbours(t, mark, nb);
            adj_ptr[t + 1] = (int32_t)nb.size();
            for (int32_t s : nb) {
                int sa[3], sb[3], ns = 0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        if (T[3 * t + a] == T[3 * (int64_t)s + b]) {
                            sa[ns] = a;
                            sb[ns] = b;
                            ++ns;
                        }
                int pt[3], ps[3], kind;
                if (ns == 3) {
                    kind = 0;
                    for (int k = 0; k < 3; ++k) pt[k] = ps[k] = k;
                } else if (ns == 2) {
                    // shared edge from reordered vertex 0 to 1 in both, directed from its lower to its
                    // higher global index: the rule of (s, t) is then that of (t, s) with roles exchanged
                    kind = 1;
                    const int k0 = T[3 * t + sa[0]] < T[3 * t + sa[1]] ? 0 : 1, k1 = 1 - k0;
                    pt[0] = sa[k0]; pt[1] = sa[k1]; pt[2] = 3 - sa[0] - sa[1];
                    ps[0] = sb[k0]; ps[1] = sb[k1]; ps[2] = 3 - sb[0] - sb[1];
                } else {
                    kind = 2;  // shared vertex is reordered vertex 0 in both (ns == 1 by construction)
                    for (int k = 0; k < 3; ++k) {
                        pt[k] = (sa[0] + k) % 3;
                        ps[k] = (sb[0] + k) % 3;
                    }
                }
                int code = pt[0] | pt[1] << 2 | pt[2] << 4 | ps[0] << 6 | ps[1] << 8 | ps[2] << 10;
                out.push_back(make_int4((int)t, s, kind, code));
            }
        }
    });
    for (int64_t t = 0; t < nt; ++t) adj_ptr[t + 1] += adj_ptr[t];
    const int64_t n_adj = adj_ptr[nt];
    std::vector<int4> pairs(n_adj);
    {
        int64_t o = 0;
        for (int c = 0; c < nchunk; ++c) {
            std::copy(chunk_pairs[c].begin(), chunk_pairs[c].end(), pairs.begin() + o);
            o += (int64_t)chunk_pairs[c].size();
        }
    }

    tr.lap("adjacency");
    // ---- each adjacent pair's reverse; the pairs the near kernels integrate:
    // coincident ones, and one of every two reversed ones (t < s)
    m->n_adj = n_adj;
    std::vector<int32_t> rev(n_adj), coin_list, prim_list;
    std::atomic<bool> rev_ok{true};
    // primary pairs: the edge-adjacent ones first, then the vertex-adjacent ones (each class
    // is integrated by its own launch with its own rule)
    std::vector<std::vector<int32_t>> chunk_coin(MAX_HOST_THREADS), chunk_prim(MAX_HOST_THREADS),
        chunk_primv(MAX_HOST_THREADS);
    std::vector<int64_t> chunk_edge(MAX_HOST_THREADS, 0);
    const int nrc = parallel_chunks(n_adj, [&](int c, int64_t b0, int64_t b1) {
        for (int64_t p = b0; p < b1; ++p) {
            const int32_t t = pairs[p].x, u = pairs[p].y;
            const int4* bg = pairs.data() + adj_ptr[u];
            const int4* en = pairs.data() + adj_ptr[u + 1];
            const int4* q = std::lower_bound(bg, en, t, [](const int4& x, int32_t v) { return x.y < v; });
            if (q == en || q->y != t) {
                rev_ok = false;
                continue;
            }
            rev[p] = (int32_t)(q - pairs.data());
            if (t == u) {
                chunk_coin[c].push_back((int32_t)p);
            } else if (t < u) {
                if (pairs[p].z == 1) {
                    chunk_prim[c].push_back((int32_t)p);
                    chunk_edge[c] += 1;
                } else {
                    chunk_primv[c].push_back((int32_t)p);
                }
            }
        }
    });
    if (!rev_ok) return set_error(PB_EMESH, "internal: pair without reverse");
    for (int c = 0; c < nrc; ++c) {  // in pair order
        coin_list.insert(coin_list.end(), chunk_coin[c].begin(), chunk_coin[c].end());
        prim_list.insert(prim_list.end(), chunk_prim[c].begin(), chunk_prim[c].end());
        m->n_prim_edge += chunk_edge[c];
    }
    for (int c = 0; c < nrc; ++c) prim_list.insert(prim_list.end(), chunk_primv[c].begin(), chunk_primv[c].end());

    tr.lap("reverse");
    size_t tot = 0;
    PB_TRY(upload((void**)&m->verts, V.data(), sizeof(double) * 3 * nv, &tot));
    PB_TRY(upload((void**)&m->tris, T.data(), sizeof(int32_t) * 3 * nt, &tot));

    // ---- distance band: pairs sharing no vertex whose centroids are closer than
    // eta (rho_t + rho_s), rho the largest centroid-vertex distance. Centroids
    // and radii here, with the oracle's arithmetic; a uniform grid of cell size
    // 2 eta max(rho) here; the search on the device (k_band_search), which
    // lists each triangle's partners in increasing order.
    tr.lap("upload_mesh");
    m->n_band = 0;
    if (eta > 0.0) {
        std::vector<double> C(3 * nt), R(nt);
        double rmax = 0.0;
        for (int64_t t = 0; t < nt; ++t) {
            const double *p0 = &V[3 * T[3 * t]], *p1 = &V[3 * T[3 * t + 1]], *p2 = &V[3 * T[3 * t + 2]];
            double c[3];
            for (int k = 0; k < 3; ++k) c[k] = (p0[k] + p1[k] + p2[k]) / 3.0;
            double r2 = 0.0;
            const double* pp[3] = {p0, p1, p2};
            for (int a = 0; a < 3; ++a) {
                double d[3] = {pp[a][0] - c[0], pp[a][1] - c[1], pp[a][2] - c[2]};
                double q = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (q > r2) r2 = q;
            }
            for (int k = 0; k < 3; ++k) C[3 * t + k] = c[k];
            R[t] = sqrt(r2);
            rmax = std::max(rmax, R[t]);
        }
        double cell = 2.0 * eta * rmax;
        int64_t dim[3];
        for (;;) {
            int64_t cells = 1;
            for (int k = 0; k < 3; ++k) {
                dim[k] = std::max<int64_t>(1, (int64_t)((hi[k] - lo[k]) / cell) + 1);
                cells *= dim[k];
            }
            if (cells <= ((int64_t)1 << 24)) break;
            cell *= 2.0;
        }
        const int64_t ncell = dim[0] * dim[1] * dim[2];
        auto cell_of = [&](int64_t t, int k) {
            return std::min<int64_t>(dim[k] - 1, std::max<int64_t>(0, (int64_t)((C[3 * t + k] - lo[k]) / cell)));
        };
        std::vector<int32_t> cstart(ncell + 1, 0), ctri(nt), tcell(nt);
        for (int64_t t = 0; t < nt; ++t) {
            tcell[t] = (int32_t)(cell_of(t, 0) + dim[0] * (cell_of(t, 1) + dim[1] * cell_of(t, 2)));
            cstart[tcell[t] + 1]++;
        }
        for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
        {
            std::vector<int32_t> fill(cstart.begin(), cstart.end() - 1);
            for (int64_t t = 0; t < nt; ++t) ctri[fill[tcell[t]]++] = (int32_t)t;
        }
        // the prefilter's FP32 copies, centred on the box
        std::vector<float4> CR32(nt);
        double cmax = 0.0;
        for (int64_t t = 0; t < nt; ++t) {
            double c[3];
            for (int k = 0; k < 3; ++k) {
                c[k] = C[3 * t + k] - 0.5 * (lo[k] + hi[k]);
                cmax = std::max(cmax, std::fabs(c[k]));
            }
            CR32[t] = make_float4((float)c[0], (float)c[1], (float)c[2], (float)R[t]);
        }
        const float slack = (float)(4.0 * std::ldexp(std::max(cmax, rmax), -23));
        // scratch on the device: C, R, the FP32 copies, grid, counts, total
        const size_t sb = sizeof(float4) * nt + sizeof(double) * 4 * nt + sizeof(int32_t) * (ncell + 1 + 3 * nt) + 64;
        char* scratch = nullptr;
        PB_TRY(dev_alloc((void**)&scratch, sb));
        float4* dCR = (float4*)scratch;
        double* dC = (double*)(dCR + nt);
        double* dR = dC + 3 * nt;
        int64_t* dtotal = (int64_t*)(dR + nt);
        int32_t* dcs = (int32_t*)(dtotal + 1);
        int32_t* dct = dcs + ncell + 1;
        int32_t* dtc = dct + nt;
        int32_t* dcnt = dtc + nt;
        int rc = PB_OK;
        int64_t total = 0;
        do {
            if (cudaMemcpy(dCR, CR32.data(), sizeof(float4) * nt, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(dC, C.data(), sizeof(double) * 3 * nt, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(dR, R.data(), sizeof(double) * nt, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(dcs, cstart.data(), sizeof(int32_t) * (ncell + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(dct, ctri.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(dtc, tcell.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice) != cudaSuccess) {
                rc = set_error(PB_ECUDA, "band search upload failed");
                break;
            }
            BandGrid g = {dC, dR, dCR, slack, dcs, dct, dtc, {dim[0], dim[1], dim[2]}, eta};
            const unsigned nb = (unsigned)((nt * 32 + 127) / 128);  // a warp per triangle
            rc = dev_alloc((void**)&m->band_ptr, sizeof(int32_t) * (nt + 1));
            if (rc != PB_OK) break;
            k_band_search<<<nb, 128>>>(nt, m->tris, g, 0, dcnt, nullptr, nullptr, nullptr);
            k_scan<<<1, 1024>>>(nt, dcnt, m->band_ptr, dtotal);
            ::pb::count_launch(2);
            if (cudaMemcpy(&total, dtotal, sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
                rc = set_error(PB_ECUDA, "band search failed");
                break;
            }
            if (total + n_adj > (((int64_t)1 << 31) - 1) / 9) {
                rc = set_error(PB_EINVAL, "distance band too wide for this mesh (%lld pairs)", (long long)total);
                break;
            }
            m->n_band = total;
            if ((rc = dev_alloc((void**)&m->band_s, sizeof(int32_t) * (total + 1))) != PB_OK) break;
            if ((rc = dev_alloc((void**)&m->band_t, sizeof(int32_t) * (total + 1))) != PB_OK) break;
            k_band_search<<<nb, 128>>>(nt, m->tris, g, 1, nullptr, m->band_ptr, m->band_s, m->band_t);
            ::pb::count_launch();
        } while (false);
        cudaFree(scratch);
        if (rc != PB_OK) return rc;
        tot += sizeof(int32_t) * (nt + 1 + 2 * (m->n_band + 1));
    }
    m->npairs = n_adj + m->n_band;
    tr.lap("band");

    // ---- near pattern (device): counts, row pointers, sorted columns, then the
    // transposed and diagonal positions
    PB_TRY(upload((void**)&m->v2t_ptr, v2t_ptr.data(), sizeof(int32_t) * (nv + 1), &tot));
    PB_TRY(upload((void**)&m->v2t, v2t.data(), sizeof(int32_t) * 3 * nt, &tot));
    PB_TRY(upload((void**)&m->pairs, pairs.data(), sizeof(int4) * pairs.size(), &tot));
    PB_TRY(upload((void**)&m->adj_ptr, adj_ptr.data(), sizeof(int32_t) * (nt + 1), &tot));
    PB_TRY(upload((void**)&m->pair_rev, rev.data(), sizeof(int32_t) * rev.size(), &tot));
    PB_TRY(upload((void**)&m->pair_coin, coin_list.data(), sizeof(int32_t) * coin_list.size(), &tot));
    PB_TRY(upload((void**)&m->pair_prim, prim_list.data(), sizeof(int32_t) * prim_list.size(), &tot));
    m->n_coin = (int64_t)coin_list.size();
    m->n_prim = (int64_t)prim_list.size();
    tr.lap("upload_pairs");
    PB_TRY(dev_alloc((void**)&m->status, sizeof(int)));
    PB_CUDA(cudaMemset(m->status, 0, sizeof(int)));
    PB_TRY(dev_alloc((void**)&m->row_ptr, sizeof(int32_t) * (nv + 1)));
    tot += sizeof(int32_t) * (nv + 1);
    {
        int32_t* cntv = nullptr;
        PB_TRY(dev_alloc((void**)&cntv, sizeof(int32_t) * nv + 64));
        int64_t* dtot = (int64_t*)(cntv + nv + (nv & 1));
        int* dmax = (int*)(dtot + 1);
        int* dcand = dmax + 1;
        int* dovf = dmax + 2;
        int rc = PB_OK;
        int64_t nnz = 0;
        int hmax = 0, st = 0, maxc = 0;
        const int32_t* bp = m->n_band ? m->band_ptr : nullptr;
        int PAT_HASH = 0, PAT_WARPS = 1;
        size_t psmem = 0;
        unsigned pb_blocks = 0;
        do {
            if (cudaMemset(dmax, 0, 2 * sizeof(int)) != cudaSuccess) { rc = set_error(PB_ECUDA, "pattern"); break; }
            k_row_candidates<<<(unsigned)((nv + 127) / 128), 128>>>(nv, m->v2t_ptr, m->v2t, m->adj_ptr, bp, dcand);
            ::pb::count_launch();
            if (cudaMemcpy(&maxc, dcand, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
                rc = set_error(PB_ECUDA, "near pattern failed");
                break;
            }
            // hash slots: a power of two; pass 0 from 512 (or twice the candidates, if fewer) up to
            // twice the candidates (at most 32768), warps per block so that a block stays within
            // 160 KB of shared memory. The dynamic shared-memory limit is the largest allowed
            // (227 KB; a block takes at most 6 x 32768 x 4 B = 192 KB), whatever the launch
            // takes: another host thread may load a mesh at the same time, and a smaller limit
            // set by it must not stand when this launch runs.
            if (cudaFuncSetAttribute(k_row_pattern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 << 10) !=
                cudaSuccess) {
                rc = set_error(PB_ECUDA, "near pattern: shared memory refused");
                break;
            }
            int hash_cap = 64;
            while (hash_cap < 2 * maxc && hash_cap < 32768) hash_cap *= 2;
            auto shape = [&](int slots) {
                PAT_HASH = slots;
                const size_t per_warp = sizeof(int32_t) * (size_t)(PAT_HASH + PAT_HASH / 2);
                PAT_WARPS = (int)std::max<size_t>(1, std::min<size_t>(8, (160u << 10) / per_warp));
                psmem = per_warp * PAT_WARPS;
                pb_blocks = (unsigned)((nv + PAT_WARPS - 1) / PAT_WARPS);
            };
            int ovf = 0;
            for (int slots = std::min(512, hash_cap);; slots = std::min(4 * slots, hash_cap)) {
                shape(slots);
                if (cudaMemset(dmax, 0, 3 * sizeof(int)) != cudaSuccess) { rc = set_error(PB_ECUDA, "pattern"); break; }
                k_row_pattern<<<pb_blocks, 32 * PAT_WARPS, psmem>>>(nv, 0, PAT_HASH, PAT_WARPS, m->v2t_ptr, m->v2t,
                                                                     m->tris, m->adj_ptr, m->pairs, bp, m->band_s,
                                                                     cntv, dmax, nullptr, nullptr, dovf, m->status);
                ::pb::count_launch();
                if (cudaMemcpy(&ovf, dovf, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
                    rc = set_error(PB_ECUDA, "near pattern failed");
                    break;
                }
                if (!ovf || slots >= hash_cap) break;
            }
            if (rc != PB_OK) break;
            if (ovf) {
                rc = set_error(PB_EINVAL, "near pattern: a row has more than %d columns (distance band too wide)",
                               PAT_HASH / 2);
                break;
            }
            k_scan<<<1, 1024>>>(nv, cntv, m->row_ptr, dtot);
            ::pb::count_launch();
            if (cudaMemcpy(&nnz, dtot, sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(&hmax, dmax, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
                rc = set_error(PB_ECUDA, "near pattern failed");
                break;
            }
            if (st != 0) {
                rc = set_error(PB_EINVAL, "near pattern: a row has more than %d columns (distance band too wide)",
                               PAT_HASH / 2);
                break;
            }
            if (nnz > ((int64_t)1 << 31) - 1) {
                rc = set_error(PB_EINVAL, "near pattern too large");
                break;
            }
            m->nnz = nnz;
            m->max_row = hmax;
            if ((rc = dev_alloc((void**)&m->col, sizeof(int32_t) * (nnz + 1))) != PB_OK) break;
            // every row has at most hmax columns: a set of twice that many slots holds any of them
            int slots1 = 64;
            while (slots1 < 2 * hmax && slots1 < 32768) slots1 *= 2;
            shape(std::min(slots1, PAT_HASH));
            k_row_pattern<<<pb_blocks, 32 * PAT_WARPS, psmem>>>(nv, 1, PAT_HASH, PAT_WARPS, m->v2t_ptr, m->v2t,
                                                                 m->tris, m->adj_ptr, m->pairs, bp, m->band_s, nullptr,
                                                                 nullptr, m->row_ptr, m->col, dovf, m->status);
            ::pb::count_launch();
        } while (false);
        cudaFree(cntv);
        if (rc != PB_OK) return rc;
    }
    tr.lap("pattern");
    const int64_t nnz = m->nnz;
    PB_TRY(dev_alloc((void**)&m->tpos, sizeof(int32_t) * nnz));
    PB_TRY(dev_alloc((void**)&m->row_of, sizeof(int32_t) * nnz));
    PB_TRY(dev_alloc((void**)&m->diag_pos, sizeof(int32_t) * nv));
    tot += sizeof(int32_t) * (3 * nnz + nv);
    k_pattern_maps<<<(unsigned)((nv * 32 + 127) / 128), 128>>>(nv, m->row_ptr, m->col, m->tpos, m->diag_pos, m->row_of,
                                                          m->status);
    ::pb::count_launch();
    PB_TRY(dev_alloc((void**)&m->tgeo, sizeof(double) * 16 * nt));
    PB_TRY(dev_alloc((void**)&m->pts64, sizeof(double) * 4 * m->np));
    PB_TRY(dev_alloc((void**)&m->pts32, sizeof(float) * 4 * m->np));
    PB_TRY(dev_alloc((void**)&m->pts32lo, sizeof(float) * 4 * m->np));
    tot += sizeof(double) * 16 * nt + (sizeof(double) + 2 * sizeof(float)) * 4 * m->np;
    m->np_ref = nt * m->Qr;
    if (m->Qr != m->Q) {
        PB_TRY(dev_alloc((void**)&m->pts_ref, sizeof(double) * 4 * m->np_ref));
        tot += sizeof(double) * 4 * m->np_ref;
    } else {
        m->pts_ref = m->pts64;
    }
    m->device_bytes = tot;

    double cx = 0.5 * (lo[0] + hi[0]), cy = 0.5 * (lo[1] + hi[1]), cz = 0.5 * (lo[2] + hi[2]);
    m->ctr[0] = cx;
    m->ctr[1] = cy;
    m->ctr[2] = cz;
    int threads = 128;
    int blocks = (int)((nt + threads - 1) / threads);
    k_geometry<<<blocks, threads>>>(m->verts, m->tris, nt, mesh_rule(m), mesh_ref_rule(m), cx, cy, cz, m->tgeo,
                                    m->pts64, m->pts32, m->pts32lo, m->pts_ref != m->pts64 ? m->pts_ref : nullptr);
    ::pb::count_launch();
    PB_CUDA(cudaGetLastError());
    PB_CUDA(cudaDeviceSynchronize());
    int st = 0;
    PB_CUDA(cudaMemcpy(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) return set_error(PB_EMESH, "internal: near pattern is not symmetric");
    tr.lap("geometry");
    return PB_OK;
}

}  // namespace pb

using namespace pb;

extern "C" int pb_mesh_load(pb_ctx* ctx, const double* verts, int64_t n_verts, const int32_t* tris,
                            int64_t n_tris, const pb_quad_plan* plan, int mem, pb_mesh** out) {
    if (!ctx || !verts || !tris || !out) return set_error(PB_EINVAL, "pb_mesh_load: NULL argument");
    *out = nullptr;
    PB_CUDA(cudaSetDevice(ctx->device));
    pb_mesh* m = new pb_mesh();
    for (Workspace* w : {&m->ws_src, &m->ws_part, &m->ws_tri, &m->ws_vec, &m->ws_comb, &m->ws_tree}) w->gen = &m->ws_gen;
    int rc = load(ctx, verts, n_verts, tris, n_tris, plan, mem, m);
    if (rc != PB_OK) {
        free_mesh_arrays(m);
        delete m;
        return rc;
    }
    *out = m;
    return PB_OK;
}

extern "C" int pb_free_mesh(pb_mesh* m) {
    if (!m) return PB_OK;
    free_mesh_arrays(m);
    delete m;
    return PB_OK;
}

extern "C" int pb_mesh_info(const pb_mesh* m, int64_t out[6]) {
    if (!m || !out) return set_error(PB_EINVAL, "pb_mesh_info: NULL argument");
    out[0] = m->nv;
    out[1] = m->nt;
    out[2] = m->np;
    out[3] = m->nnz;
    out[4] = m->npairs;
    out[5] = (int64_t)(m->device_bytes + m->ws_src.bytes + m->ws_part.bytes + m->ws_tri.bytes +
                       m->ws_vec.bytes + m->ws_comb.bytes);
    return PB_OK;
}
