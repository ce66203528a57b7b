// a1: mesh ingest - validation, topology, quadrature points, adjacent
// triangle pairs and the vertex-pair pattern of the near field.
//
// Paper, "Numerical discretization": continuous piecewise-linear Galerkin
// elements on a triangular surface mesh, one unknown per vertex. Far
// (non-adjacent) triangle pairs are integrated with one symmetric triangle
// rule on both triangles; pairs that share a vertex are singular and get the
// regularised rule of the near field (near.cu).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

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
                           int64_t nt, Rule rule, double cx, double cy, double cz,
                           double* __restrict__ tgeo, double* __restrict__ pts64,
                           float* __restrict__ pts32, float* __restrict__ pts32lo) {
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
}

static int upload(void** dst, const void* src, size_t bytes, size_t* total) {
    PB_TRY(dev_alloc(dst, bytes));
    if (bytes) PB_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    *total += bytes;
    return PB_OK;
}

static void free_mesh_arrays(pb_mesh* m) {
    void* ptrs[] = {m->verts, m->tris,  m->tgeo, m->pts64,    m->pts32,       m->pts32lo,
                    m->v2t_ptr, m->v2t, m->pairs, m->row_ptr, m->col,         m->tpos,
                    m->diag_pos, m->contrib_ptr, m->contrib, m->status, m->pair_rev,
                    m->pair_coin, m->pair_prim};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    ws_free(m->ws_src);
    ws_free(m->ws_part);
    ws_free(m->ws_tri);
    ws_free(m->ws_vec);
    ws_free(m->ws_comb);
}

static int load(pb_ctx* ctx, const double* verts_in, int64_t nv, const int32_t* tris_in, int64_t nt,
                const pb_quad_plan* plan, int mem, pb_mesh* m) {
    if (nv < 4 || nt < 4) return set_error(PB_EMESH, "mesh too small (%lld verts, %lld tris)",
                                           (long long)nv, (long long)nt);
    if (nt > (int64_t)1 << 28 || nv > (int64_t)1 << 28)
        return set_error(PB_EINVAL, "mesh too large for 32-bit indices");
    int Q = plan ? plan->far_q : 6;
    int nss = plan ? plan->n_ss : 4;
    if (Q != 1 && Q != 3 && Q != 6) return set_error(PB_EINVAL, "far_q must be 1, 3 or 6 (got %d)", Q);
    if (nss < 1 || nss > 12) return set_error(PB_EINVAL, "n_ss must be in 1..12 (got %d)", nss);
    m->ctx = ctx;
    m->nv = nv;
    m->nt = nt;
    m->Q = Q;
    m->n_ss = nss;
    m->np = nt * Q;
    rule_points(Q, m->rule_l, m->rule_w);

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
    // every undirected edge must appear exactly twice, once in each direction
    {
        std::vector<std::pair<uint64_t, int>> e;
        e.reserve(3 * nt);
        for (int64_t t = 0; t < nt; ++t)
            for (int a = 0; a < 3; ++a) {
                uint64_t i = T[3 * t + a], j = T[3 * t + (a + 1) % 3];
                uint64_t key = i < j ? (i << 32 | j) : (j << 32 | i);
                e.push_back({key, i < j ? 1 : -1});
            }
        std::sort(e.begin(), e.end());
        for (size_t k = 0; k < e.size();) {
            size_t l = k;
            int s = 0;
            while (l < e.size() && e[l].first == e[k].first) s += e[l++].second;
            if (l - k != 2)
                return set_error(PB_EMESH, "edge (%llu,%llu) is shared by %zu triangles (mesh not closed "
                                 "or not manifold)", (unsigned long long)(e[k].first >> 32),
                                 (unsigned long long)(e[k].first & 0xffffffffu), l - k);
            if (s != 0)
                return set_error(PB_EMESH, "edge (%llu,%llu) has the same direction in both triangles "
                                 "(inconsistent orientation)", (unsigned long long)(e[k].first >> 32),
                                 (unsigned long long)(e[k].first & 0xffffffffu));
            k = l;
        }
    }
    if (!(vol6 > 0.0))
        return set_error(PB_EMESH, "enclosed volume is not positive (triangles must be counter-clockwise "
                         "seen from outside)");

    // ---- vertex -> triangle map
    std::vector<int32_t> v2t_ptr(nv + 1, 0), v2t(3 * nt);
    for (int64_t k = 0; k < 3 * nt; ++k) v2t_ptr[T[k] + 1]++;
    for (int64_t i = 0; i < nv; ++i) v2t_ptr[i + 1] += v2t_ptr[i];
    {
        std::vector<int32_t> fill(v2t_ptr.begin(), v2t_ptr.end() - 1);
        for (int64_t t = 0; t < nt; ++t)
            for (int a = 0; a < 3; ++a) v2t[fill[T[3 * t + a]]++] = (int32_t)(3 * t + a);
    }
    for (int64_t i = 0; i < nv; ++i)
        if (v2t_ptr[i + 1] == v2t_ptr[i])
            return set_error(PB_EMESH, "vertex %lld belongs to no triangle", (long long)i);

    // ---- adjacent triangle pairs (share >= 1 vertex), ordered by (ti, tj)
    std::vector<int4> pairs;
    pairs.reserve(16 * nt);
    {
        std::vector<int32_t> mark(nt, -1);
        std::vector<int32_t> nb;
        for (int64_t t = 0; t < nt; ++t) {
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
                } else if (ns == 1) {
                    kind = 2;  // shared vertex is reordered vertex 0 in both
                    for (int k = 0; k < 3; ++k) {
                        pt[k] = (sa[0] + k) % 3;
                        ps[k] = (sb[0] + k) % 3;
                    }
                } else {
                    return set_error(PB_EMESH, "internal: neighbour without a shared vertex");
                }
                int code = pt[0] | pt[1] << 2 | pt[2] << 4 | ps[0] << 6 | ps[1] << 8 | ps[2] << 10;
                pairs.push_back(make_int4((int)t, s, kind, code));
            }
        }
    }
    m->npairs = (int64_t)pairs.size();

    // ---- near pattern: row i holds every vertex of every triangle adjacent to a
    // triangle at i (the 2-ring); built with a marker array, then sorted.
    std::vector<int32_t> pair_ptr(nt + 1, 0);
    for (const int4& p : pairs) pair_ptr[p.x + 1]++;
    for (int64_t t = 0; t < nt; ++t) pair_ptr[t + 1] += pair_ptr[t];
    // each ordered pair's reverse, and the pairs the near kernel integrates:
    // coincident ones, and one of every two reversed ones (t < s)
    std::vector<int32_t> rev(pairs.size()), coin_list, prim_list;
    for (size_t p = 0; p < pairs.size(); ++p) {
        const int32_t t = pairs[p].x, u = pairs[p].y;
        int32_t lo = pair_ptr[u], hi = pair_ptr[u + 1];
        while (lo < hi) {
            int32_t mid = (lo + hi) / 2;
            if (pairs[mid].y < t) lo = mid + 1;
            else hi = mid;
        }
        if (lo >= pair_ptr[u + 1] || pairs[lo].y != t) return set_error(PB_EMESH, "internal: pair without reverse");
        rev[p] = lo;
        if (t == u) coin_list.push_back((int32_t)p);
        else if (t < u) prim_list.push_back((int32_t)p);
    }
    std::vector<int32_t> row_ptr(nv + 1, 0), col, mark(nv, -1), colpos(nv, 0);
    col.reserve((size_t)24 * nv);
    for (int64_t i = 0; i < nv; ++i) {
        size_t start = col.size();
        for (int32_t k = v2t_ptr[i]; k < v2t_ptr[i + 1]; ++k) {
            int32_t t = v2t[k] / 3;
            for (int32_t p = pair_ptr[t]; p < pair_ptr[t + 1]; ++p) {
                const int32_t* f = &T[3 * (int64_t)pairs[p].y];
                for (int b = 0; b < 3; ++b)
                    if (mark[f[b]] != (int32_t)i) {
                        mark[f[b]] = (int32_t)i;
                        col.push_back(f[b]);
                    }
            }
        }
        std::sort(col.begin() + start, col.end());
        if (col.size() > (size_t)(((int64_t)1 << 31) - 1)) return set_error(PB_EINVAL, "near pattern too large");
        row_ptr[i + 1] = (int32_t)col.size();
    }
    const int64_t nnz = (int64_t)col.size();
    m->nnz = nnz;
    std::vector<int32_t> tpos(nnz), diag_pos(nv, -1);
    for (int64_t i = 0; i < nv; ++i)
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            const int32_t j = col[k];
            const int32_t* bg = col.data() + row_ptr[j];
            const int32_t* en = col.data() + row_ptr[j + 1];
            const int32_t* q = std::lower_bound(bg, en, (int32_t)i);
            if (q == en || *q != (int32_t)i) return set_error(PB_EMESH, "internal: near pattern is not symmetric");
            tpos[k] = (int32_t)(q - col.data());
            if (j == i) diag_pos[i] = k;
        }

    // ---- contributions (pair * 9 + a * 3 + b) of every adjacent pair to each
    // nonzero, listed row by row in a fixed order (corners of the row vertex,
    // then its triangle's pairs, then the trial corner): a counting pass and a
    // filling pass over the same loops.
    std::vector<int32_t> cnt(nnz + 1, 0);
    std::vector<int32_t> cidx((size_t)9 * pairs.size());
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<int32_t> fill;
        if (pass == 1) {
            for (int64_t k = 0; k < nnz; ++k) cnt[k + 1] += cnt[k];
            fill.assign(cnt.begin(), cnt.end() - 1);
        }
        for (int64_t i = 0; i < nv; ++i) {
            for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) colpos[col[k]] = k;
            for (int32_t k = v2t_ptr[i]; k < v2t_ptr[i + 1]; ++k) {
                const int32_t t = v2t[k] / 3, a = v2t[k] % 3;
                for (int32_t p = pair_ptr[t]; p < pair_ptr[t + 1]; ++p) {
                    const int32_t* f = &T[3 * (int64_t)pairs[p].y];
                    for (int b = 0; b < 3; ++b) {
                        const int32_t kk = colpos[f[b]];
                        if (pass == 0) cnt[kk + 1]++;
                        else cidx[fill[kk]++] = 9 * p + 3 * a + b;
                    }
                }
            }
        }
    }
    m->ncontrib = (int64_t)cidx.size();

    // ---- upload
    size_t tot = 0;
    PB_TRY(upload((void**)&m->verts, V.data(), sizeof(double) * 3 * nv, &tot));
    PB_TRY(upload((void**)&m->tris, T.data(), sizeof(int32_t) * 3 * nt, &tot));
    PB_TRY(upload((void**)&m->v2t_ptr, v2t_ptr.data(), sizeof(int32_t) * (nv + 1), &tot));
    PB_TRY(upload((void**)&m->v2t, v2t.data(), sizeof(int32_t) * 3 * nt, &tot));
    PB_TRY(upload((void**)&m->pairs, pairs.data(), sizeof(int4) * pairs.size(), &tot));
    PB_TRY(upload((void**)&m->pair_rev, rev.data(), sizeof(int32_t) * rev.size(), &tot));
    PB_TRY(upload((void**)&m->pair_coin, coin_list.data(), sizeof(int32_t) * coin_list.size(), &tot));
    PB_TRY(upload((void**)&m->pair_prim, prim_list.data(), sizeof(int32_t) * prim_list.size(), &tot));
    m->n_coin = (int64_t)coin_list.size();
    m->n_prim = (int64_t)prim_list.size();
    PB_TRY(upload((void**)&m->row_ptr, row_ptr.data(), sizeof(int32_t) * (nv + 1), &tot));
    PB_TRY(upload((void**)&m->col, col.data(), sizeof(int32_t) * nnz, &tot));
    PB_TRY(upload((void**)&m->tpos, tpos.data(), sizeof(int32_t) * nnz, &tot));
    PB_TRY(upload((void**)&m->diag_pos, diag_pos.data(), sizeof(int32_t) * nv, &tot));
    PB_TRY(upload((void**)&m->contrib_ptr, cnt.data(), sizeof(int32_t) * (nnz + 1), &tot));
    PB_TRY(upload((void**)&m->contrib, cidx.data(), sizeof(int32_t) * cidx.size(), &tot));
    PB_TRY(dev_alloc((void**)&m->status, sizeof(int)));
    PB_CUDA(cudaMemset(m->status, 0, sizeof(int)));
    PB_TRY(dev_alloc((void**)&m->tgeo, sizeof(double) * 16 * nt));
    PB_TRY(dev_alloc((void**)&m->pts64, sizeof(double) * 4 * m->np));
    PB_TRY(dev_alloc((void**)&m->pts32, sizeof(float) * 4 * m->np));
    PB_TRY(dev_alloc((void**)&m->pts32lo, sizeof(float) * 4 * m->np));
    tot += sizeof(double) * 16 * nt + (sizeof(double) + 2 * sizeof(float)) * 4 * m->np;
    m->device_bytes = tot;

    double cx = 0.5 * (lo[0] + hi[0]), cy = 0.5 * (lo[1] + hi[1]), cz = 0.5 * (lo[2] + hi[2]);
    int threads = 128;
    int blocks = (int)((nt + threads - 1) / threads);
    k_geometry<<<blocks, threads>>>(m->verts, m->tris, nt, mesh_rule(m), cx, cy, cz, m->tgeo, m->pts64, m->pts32,
                                    m->pts32lo); ::pb::count_launch();
    PB_CUDA(cudaGetLastError());
    PB_CUDA(cudaDeviceSynchronize());
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
