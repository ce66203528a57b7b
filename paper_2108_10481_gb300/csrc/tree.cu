// Treecode far field for the FP32 inner iterations: a fast far field in place
// of the direct pair sum for large meshes, where the paper uses a fast
// multipole method (ExaFMM, expansion order 3).
//
// The quadrature points are sorted into a kd-tree (longest-axis splits near
// the median, with a multiple of TREE_LEAF points on the left, so that the
// leaves hold TREE_LEAF points but one per path). For a leaf of targets and a cluster
// that is well separated (radius sum below theta times the centre distance),
// the cluster's sources are replaced by proxy sources on an n x n x n tensor
// grid of Chebyshev points of its bounding box: the y-dependence of every
// kernel is interpolated by the tensor Lagrange basis L_k, so
//   sum_j G(x, y_j) s_j            ~ sum_k G(x, z_k) S_k,     S_k = sum_j L_k(y_j) s_j
//   sum_j grad_y G(x, y_j) . p_j   ~ sum_k G(x, z_k) Q_k,     Q_k = sum_j grad L_k(y_j) . p_j
//   sum_j grad_x G(x, y_j) s_j     ~ sum_k grad_x G(x, z_k) S_k
// and the vector charges (curl densities, normal densities) likewise, for
// both kernels at once (the interpolation is kernel independent). Clusters
// with fewer points than proxies, and all other pairs, are summed directly
// with the same arithmetic as the direct FP32 pair kernel (identical points
// skipped; the direct and proxy arithmetic is the same formula with the
// charges that only meet constant coefficients combined with them once per
// staged record). The result approximates the direct far sum; the mixed-precision
// solver uses it only for its inner iterations and keeps the exact sums for
// the outer residual.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "tree_eval.cuh"

namespace pb {

constexpr int TREE_MAXN = 8;        // largest Chebyshev order + 1
constexpr int TREE_MAX_SPLITS = 8;  // CTAs sharing one leaf's interaction lists

// ---------------------------------------------------------------- host tree
struct HostNode {
    float lo[3], hi[3];
    int32_t b, e;     // points [b, e) in tree order
    int32_t c0, c1;   // children (-1 for a leaf)
    int32_t proxy;    // proxy slot (-1: fewer points than proxies)
};

struct PbTree {
    int n = 0, nprox = 0;       // Chebyshev points per dimension, proxies per cluster
    double theta = 0.0;
    int64_t nleaf = 0, nslot = 0;
    int32_t* perm = nullptr;      // tree index -> point index
    int32_t* leaf_rng = nullptr;  // 2 per leaf
    int32_t* leaf_order = nullptr;// leaves by decreasing interaction count (launch order)
    int32_t* far_ptr = nullptr;   // nleaf + 1
    int32_t* far_idx = nullptr;   // proxy slots
    int32_t* near_ptr = nullptr;  // nleaf + 1
    int32_t* near_rng = nullptr;  // 2 per entry: [b, e) in tree order
    int32_t* slot_rng = nullptr;  // 2 per proxy slot: its points [b, e)
    int32_t* slot_kids = nullptr; // 6 per proxy slot: per child, its slot (-1: none) and points [b, e)
    int32_t* slot_order = nullptr;// slots by height (children before parents)
    std::vector<int64_t> height_ptr;  // slot_order ranges of each height
    float* slot_box = nullptr;    // 6 per proxy slot: lo, hi
    void* block = nullptr;        // one allocation holding the arrays above
    int64_t n_far = 0, n_near = 0, direct_pairs = 0, proxy_pairs = 0;
};

void tree_free(PbTree* t) {
    if (!t) return;
    if (t->block) cudaFree(t->block);
    delete t;
}

static int build_tree(pb_mesh* m, int order, double theta, PbTree** out) {
    const int64_t np = m->np;
    std::vector<float> P(4 * np);
    PB_CUDA(cudaMemcpy(P.data(), m->pts32, sizeof(float) * 4 * np, cudaMemcpyDeviceToHost));
    std::vector<int32_t> perm(np);
    std::iota(perm.begin(), perm.end(), 0);
    std::vector<HostNode> nodes;
    nodes.reserve(2 * np / TREE_LEAF + 16);
    const int n = order + 1, nprox = n * n * n;
    // recursive split on the longest axis (explicit stack), near the median but with a multiple of
    // TREE_LEAF points on the left: every leaf then holds TREE_LEAF points but at most one per
    // path, and the evaluation's f32x2 lanes (a thread's targets i and i + TREE_LEAF / 2) are full
    // (median splits leave 81 points per leaf on average on the 5,000-atom molecule)
    struct Job { int32_t b, e, node; };
    nodes.push_back(HostNode{});
    std::vector<Job> stack{{0, (int32_t)np, 0}};
    while (!stack.empty()) {
        Job j = stack.back();
        stack.pop_back();
        HostNode nd;
        for (int k = 0; k < 3; ++k) {
            nd.lo[k] = INFINITY;
            nd.hi[k] = -INFINITY;
        }
        for (int32_t i = j.b; i < j.e; ++i)
            for (int k = 0; k < 3; ++k) {
                nd.lo[k] = std::min(nd.lo[k], P[4 * perm[i] + k]);
                nd.hi[k] = std::max(nd.hi[k], P[4 * perm[i] + k]);
            }
        nd.b = j.b;
        nd.e = j.e;
        nd.c0 = nd.c1 = -1;
        nd.proxy = -1;
        if (j.e - j.b > TREE_LEAF) {
            int ax = 0;
            for (int k = 1; k < 3; ++k)
                if (nd.hi[k] - nd.lo[k] > nd.hi[ax] - nd.lo[ax]) ax = k;
            const int32_t n_here = j.e - j.b, half = n_here / 2;
            const int32_t mid = j.b + std::min(n_here - 1, (half + TREE_LEAF - 1) / TREE_LEAF * TREE_LEAF);
            std::nth_element(perm.begin() + j.b, perm.begin() + mid, perm.begin() + j.e,
                             [&](int32_t a, int32_t c) { return P[4 * a + ax] < P[4 * c + ax]; });
            nd.c0 = (int32_t)nodes.size();
            nodes.push_back(HostNode{});
            nd.c1 = (int32_t)nodes.size();
            nodes.push_back(HostNode{});
            stack.push_back({mid, j.e, nd.c1});
            stack.push_back({j.b, mid, nd.c0});
        }
        nodes[j.node] = nd;
    }
    // proxy slots: clusters with more points than proxies
    std::vector<int32_t> slot_rng, leaves;
    std::vector<float> slot_box;
    for (size_t k = 0; k < nodes.size(); ++k) {
        HostNode& nd = nodes[k];
        if (nd.e - nd.b > nprox) {
            nd.proxy = (int32_t)(slot_rng.size() / 2);
            slot_rng.push_back(nd.b);
            slot_rng.push_back(nd.e);
            // a box with room around degenerate sides, so that the Chebyshev points are distinct
            float ext = 0.f;
            for (int d = 0; d < 3; ++d) ext = std::max(ext, nd.hi[d] - nd.lo[d]);
            for (int d = 0; d < 3; ++d) {
                const float pad = std::max(1e-3f * ext, 1e-6f);
                slot_box.push_back(nd.lo[d] - pad);
            }
            for (int d = 0; d < 3; ++d) {
                const float pad = std::max(1e-3f * ext, 1e-6f);
                slot_box.push_back(nd.hi[d] + pad);
            }
        }
        if (nd.c0 < 0) leaves.push_back((int32_t)k);
    }
    // children of every slot, and the slots ordered by height so that children's proxies exist
    // before their parents'. A slot that is a leaf (fewer points per leaf than proxies) takes
    // its own points as one raw child.
    const int64_t nslot = (int64_t)(slot_rng.size() / 2);
    std::vector<int32_t> slot_kids(6 * nslot), height(nslot, 0), slot_node(nslot);
    for (size_t k = 0; k < nodes.size(); ++k)
        if (nodes[k].proxy >= 0) slot_node[nodes[k].proxy] = (int32_t)k;
    // nodes were created parents before children: a reverse sweep sees children first
    for (int64_t sl = nslot - 1; sl >= 0; --sl) {
        const HostNode& nd = nodes[slot_node[sl]];
        if (nd.c0 < 0) {
            const int32_t own[6] = {-1, nd.b, nd.e, -1, nd.e, nd.e};
            for (int c = 0; c < 6; ++c) slot_kids[6 * sl + c] = own[c];
            height[sl] = 0;
            continue;
        }
        const int32_t kids[2] = {nd.c0, nd.c1};
        int h = 0;
        for (int c = 0; c < 2; ++c) {
            const HostNode& ch = nodes[kids[c]];
            slot_kids[6 * sl + 3 * c] = ch.proxy;
            slot_kids[6 * sl + 3 * c + 1] = ch.b;
            slot_kids[6 * sl + 3 * c + 2] = ch.e;
            if (ch.proxy >= 0) h = std::max(h, height[ch.proxy] + 1);
        }
        height[sl] = h;
    }
    auto center_radius = [&](const HostNode& nd, float* c) {
        float r2 = 0.f;
        for (int d = 0; d < 3; ++d) {
            c[d] = 0.5f * (nd.lo[d] + nd.hi[d]);
            const float h = 0.5f * (nd.hi[d] - nd.lo[d]);
            r2 += h * h;
        }
        return std::sqrt(r2);
    };
    // interaction lists of every leaf
    std::vector<int32_t> far_ptr{0}, far_idx, near_ptr{0}, near_rng, leaf_rng;
    PbTree* t = new PbTree();
    t->n = n;
    t->nprox = nprox;
    t->theta = theta;
    std::vector<int32_t> st;
    for (int32_t L : leaves) {
        const HostNode& tl = nodes[L];
        float cl[3];
        const float rl = center_radius(tl, cl);
        leaf_rng.push_back(tl.b);
        leaf_rng.push_back(tl.e);
        st.assign(1, 0);
        while (!st.empty()) {
            const HostNode& nd = nodes[st.back()];
            st.pop_back();
            float cn[3];
            const float rn = center_radius(nd, cn);
            float d2 = 0.f;
            for (int d = 0; d < 3; ++d) d2 += (cl[d] - cn[d]) * (cl[d] - cn[d]);
            const float lim = (rl + rn) / (float)theta;
            const bool separated = d2 > lim * lim;
            if (separated && nd.proxy >= 0) {
                far_idx.push_back(nd.proxy);
                t->proxy_pairs += (int64_t)(tl.e - tl.b) * nprox;
            } else if (separated || nd.c0 < 0) {
                near_rng.push_back(nd.b);
                near_rng.push_back(nd.e);
                t->direct_pairs += (int64_t)(tl.e - tl.b) * (nd.e - nd.b);
            } else {
                st.push_back(nd.c1);
                st.push_back(nd.c0);
            }
        }
        far_ptr.push_back((int32_t)far_idx.size());
        near_ptr.push_back((int32_t)(near_rng.size() / 2));
    }
    // launch order: the leaves with the most interactions first, so that the CTAs the scheduler
    // hands out last are the short ones (longest-first list scheduling)
    std::vector<int64_t> cost(leaves.size(), 0);
    for (size_t l = 0; l < leaves.size(); ++l) {
        int64_t c = (int64_t)(far_ptr[l + 1] - far_ptr[l]) * nprox;
        for (int32_t k = near_ptr[l]; k < near_ptr[l + 1]; ++k) c += near_rng[2 * k + 1] - near_rng[2 * k];
        cost[l] = c * (leaf_rng[2 * l + 1] - leaf_rng[2 * l]);
    }
    std::vector<int32_t> leaf_order(leaves.size());
    std::iota(leaf_order.begin(), leaf_order.end(), 0);
    std::stable_sort(leaf_order.begin(), leaf_order.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
    // the slots whose proxies are read: those in a far list, and (for the transfer) every slot
    // below one of them; parents have lower slot numbers than their children
    std::vector<char> needed(nslot, 0);
    for (int32_t f : far_idx) needed[f] = 1;
    for (int64_t sl = 0; sl < nslot; ++sl)
        if (needed[sl])
            for (int c = 0; c < 2; ++c)
                if (slot_kids[6 * sl + 3 * c] >= 0) needed[slot_kids[6 * sl + 3 * c]] = 1;
    int hmax = 0;
    for (int64_t sl = 0; sl < nslot; ++sl) hmax = std::max(hmax, height[sl]);
    std::vector<int32_t> slot_order;
    std::vector<int64_t> height_ptr{0};
    for (int h = 0; h <= hmax && nslot; ++h) {
        for (int64_t sl = 0; sl < nslot; ++sl)
            if (height[sl] == h && needed[sl]) slot_order.push_back((int32_t)sl);
        if ((int64_t)slot_order.size() > height_ptr.back()) height_ptr.push_back((int64_t)slot_order.size());
    }
    t->nleaf = (int64_t)leaves.size();
    t->nslot = (int64_t)(slot_rng.size() / 2);
    t->n_far = (int64_t)far_idx.size();
    t->n_near = (int64_t)(near_rng.size() / 2);
    // one device allocation for all arrays
    const size_t ints = perm.size() + leaf_rng.size() + leaf_order.size() + far_ptr.size() + far_idx.size() +
                        near_ptr.size() + near_rng.size() + slot_rng.size() + slot_kids.size() + slot_order.size();
    const size_t bytes = sizeof(int32_t) * (ints + 8) + sizeof(float) * (slot_box.size() + 4);
    int rc = dev_alloc(&t->block, bytes);
    if (rc != PB_OK) {
        delete t;
        return rc;
    }
    int32_t* p = (int32_t*)t->block;
    auto put = [&](const std::vector<int32_t>& v) {
        int32_t* at = p;
        if (!v.empty()) cudaMemcpy(at, v.data(), sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice);
        p += v.size();
        return at;
    };
    t->perm = put(perm);
    t->leaf_rng = put(leaf_rng);
    t->leaf_order = put(leaf_order);
    t->far_ptr = put(far_ptr);
    t->far_idx = put(far_idx);
    t->near_ptr = put(near_ptr);
    t->near_rng = put(near_rng);
    t->slot_rng = put(slot_rng);
    t->slot_kids = put(slot_kids);
    t->slot_order = put(slot_order);
    t->height_ptr = height_ptr;
    t->slot_box = (float*)p;
    if (!slot_box.empty())
        cudaMemcpy(t->slot_box, slot_box.data(), sizeof(float) * slot_box.size(), cudaMemcpyHostToDevice);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        tree_free(t);
        return set_error(PB_ECUDA, "tree upload: %s", cudaGetErrorString(e));
    }
    *out = t;
    return PB_OK;
}

// ------------------------------------------------------------- device side
// Source records in tree order: position (FP32, relative to the mesh centre),
// s = w v, p = w u n, c = w curl u (the direct kernel's densities), 0, 0.
__global__ void k_tree_sources(int64_t np, int Q, Rule rule, const int32_t* __restrict__ perm,
                               const int32_t* __restrict__ tris, const double* __restrict__ tgeo,
                               const double* __restrict__ pts64, const float* __restrict__ pts32,
                               const double* __restrict__ u, const double* __restrict__ v, int need_u, int need_v,
                               float* __restrict__ rec) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    const int64_t pt = perm[i], t = pt / Q;
    const int q = (int)(pt - t * Q);
    const double* g = tgeo + 16 * t;
    const int32_t i0 = tris[3 * t], i1 = tris[3 * t + 1], i2 = tris[3 * t + 2];
    double ua[3] = {0, 0, 0}, va[3] = {0, 0, 0};
    if (need_u) { ua[0] = u[i0]; ua[1] = u[i1]; ua[2] = u[i2]; }
    if (need_v) { va[0] = v[i0]; va[1] = v[i1]; va[2] = v[i2]; }
    const double inv2a = -1.0 / (2.0 * g[3]);
    const double w = pts64[4 * pt + 3] * 0.07957747154594767;  // weight / (4 pi)
    const double uq = rule.l[q][0] * ua[0] + rule.l[q][1] * ua[1] + rule.l[q][2] * ua[2];
    const double vq = rule.l[q][0] * va[0] + rule.l[q][1] * va[1] + rule.l[q][2] * va[2];
    float val[TREE_REC];
    val[0] = pts32[4 * pt];
    val[1] = pts32[4 * pt + 1];
    val[2] = pts32[4 * pt + 2];
    val[3] = (float)(w * vq);
    for (int k = 0; k < 3; ++k) val[4 + k] = (float)(w * uq * g[k]);
    for (int k = 0; k < 3; ++k)
        val[7 + k] = (float)(w * inv2a * (ua[0] * g[4 + k] + ua[1] * g[7 + k] + ua[2] * g[10 + k]));
    val[10] = val[11] = 0.f;
    float4* r = reinterpret_cast<float4*>(rec + TREE_REC * i);
    for (int k = 0; k < TREE_REC / 4; ++k) r[k] = make_float4(val[4 * k], val[4 * k + 1], val[4 * k + 2], val[4 * k + 3]);
}

// Chebyshev points (second kind) of order n-1 on [-1, 1]
__device__ __forceinline__ float cheb_node(int a, int n) {
    return cospif((float)a / (float)(n - 1));
}

// Lagrange basis l_a(t) and its derivative on the N Chebyshev points tn,
// t in [-1, 1]; iden[a] = 1 / prod_{b != a} (tn[a] - tn[b]).
template <int N>
__device__ __forceinline__ void lagrange_n(float t, const float* tn, const float* iden, float* l, float* dl) {
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float num = 1.f, dnum = 0.f;
#pragma unroll
        for (int b = 0; b < N; ++b) {
            if (b == a) continue;
            // product rule, running: d(num * (t - t_b)) = dnum (t - t_b) + num
            dnum = dnum * (t - tn[b]) + num;
            num *= t - tn[b];
        }
        l[a] = num * iden[a];
        dl[a] = dnum * iden[a];
    }
}

// Proxy charges of the slots of one height: one CTA per slot, threads over
// proxies, N Chebyshev points per axis (N^3 proxies). A slot's charges come
// from its two children: a child with its own proxies passes them on through
// the slot's interpolation (exact, the basis polynomials having the same
// degree), any other child through its points. Sources are staged 128 at a
// time with their 1-D basis values.
// Proxy record: z (3), S, Q, C (3), N (3), 0.
constexpr int PROXY_THREADS = 128;

template <int N>
__global__ void __launch_bounds__(PROXY_THREADS)
k_proxy_charges(const int32_t* __restrict__ slots, const int32_t* __restrict__ slot_kids,
                const float* __restrict__ slot_box, const float* __restrict__ rec, float* __restrict__ prox) {
    constexpr int NP = N * N * N, N2 = N * N;
    constexpr int PER = (NP + PROXY_THREADS - 1) / PROXY_THREADS;
    // a staged point: lx, ly, lz, dlx, dly, dlz (N each), 8 charges; odd row length (no bank conflicts)
    constexpr int SBW = 6 * N + 9;
    constexpr int SB = PROXY_THREADS * SBW > 2 * NP * 8 ? PROXY_THREADS * SBW : 2 * NP * 8;
    __shared__ __align__(16) float sb[SB];
    __shared__ float tn[N], iden[N];
    __shared__ float T[3][N][N];  // 1-D transfer matrices of a child with proxies
    const int slot = slots[blockIdx.x];
    if (threadIdx.x < N) tn[threadIdx.x] = cheb_node(threadIdx.x, N);
    __syncthreads();
    if (threadIdx.x < N) {
        float den = 1.f;
        for (int b = 0; b < N; ++b)
            if (b != (int)threadIdx.x) den *= tn[threadIdx.x] - tn[b];
        iden[threadIdx.x] = 1.f / den;
    }
    const float* box = slot_box + 6 * slot;
    float mid[3], half[3], ihalf[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        mid[d] = 0.5f * (box[d] + box[3 + d]);
        half[d] = 0.5f * (box[3 + d] - box[d]);
        ihalf[d] = 1.f / half[d];
    }
    // this thread's proxies and their grid indices
    int ka[PER], kb[PER], kc[PER];
    float acc[PER][8];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int k = min((int)threadIdx.x + r * PROXY_THREADS, NP - 1);
        ka[r] = k / N2;
        kb[r] = (k / N) % N;
        kc[r] = k % N;
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
    }
    __syncthreads();
    float* buf0 = sb;                // child charges, then the y pass
    float* buf1 = sb + NP * 8;       // the x pass
    for (int kid = 0; kid < 2; ++kid) {
        const int32_t ks = slot_kids[6 * slot + 3 * kid];
        if (ks >= 0) {  // uniform across the block
            // A child with proxies: its charges sit on the tensor grid of its box, so the transfer
            // to this slot's grid is a tensor product of three N x N matrices
            // T_d[a][a'] = l_a(child node a' in this slot's coordinates), applied one axis at a time.
            const float* cb = slot_box + 6 * ks;
            if (threadIdx.x < 3 * N) {
                const int d = threadIdx.x / N, a2 = threadIdx.x % N;
                const float zc = 0.5f * (cb[d] + cb[3 + d]) + 0.5f * (cb[3 + d] - cb[d]) * tn[a2];
                float l[N], dl[N];
                lagrange_n<N>((zc - mid[d]) * ihalf[d], tn, iden, l, dl);
#pragma unroll
                for (int a = 0; a < N; ++a) T[d][a][a2] = l[a];
            }
            const float* cp = prox + (int64_t)ks * NP * TREE_REC;
            for (int k = threadIdx.x; k < NP * 8; k += PROXY_THREADS) buf0[k] = cp[(k >> 3) * TREE_REC + 3 + (k & 7)];
            __syncthreads();
            for (int k = threadIdx.x; k < NP * 8; k += PROXY_THREADS) {  // x pass
                const int c = k & 7, idx = k >> 3, a = idx / N2, rest = idx - a * N2;
                float v = 0.f;
#pragma unroll
                for (int a2 = 0; a2 < N; ++a2) v += T[0][a][a2] * buf0[(a2 * N2 + rest) * 8 + c];
                buf1[k] = v;
            }
            __syncthreads();
            for (int k = threadIdx.x; k < NP * 8; k += PROXY_THREADS) {  // y pass
                const int c = k & 7, idx = k >> 3, a = idx / N2, bb = (idx / N) % N, cc = idx % N;
                float v = 0.f;
#pragma unroll
                for (int b2 = 0; b2 < N; ++b2) v += T[1][bb][b2] * buf1[((a * N + b2) * N + cc) * 8 + c];
                buf0[k] = v;
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < PER; ++r) {  // z pass into this thread's proxies
                if ((int)threadIdx.x + r * PROXY_THREADS < NP) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        float v = 0.f;
#pragma unroll
                        for (int c2 = 0; c2 < N; ++c2)
                            v += T[2][kc[r]][c2] * buf0[((ka[r] * N + kb[r]) * N + c2) * 8 + c];
                        acc[r][c] += v;
                    }
                }
            }
            __syncthreads();
            continue;
        }
        // raw points of the child: s, p (3), c (3)
        const int32_t b = slot_kids[6 * slot + 3 * kid + 1];
        const int32_t e = slot_kids[6 * slot + 3 * kid + 2];
        for (int c0 = b; c0 < e; c0 += PROXY_THREADS) {
            const int i = c0 + threadIdx.x;
            float* my = sb + threadIdx.x * SBW;
            if (i < e) {
                const float* r = rec + TREE_REC * (int64_t)i;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    lagrange_n<N>((r[d] - mid[d]) * ihalf[d], tn, iden, my + N * d, my + N * (3 + d));
#pragma unroll
                    for (int a = 0; a < N; ++a) my[N * (3 + d) + a] *= ihalf[d];  // d/dy = d/dt / half
                }
#pragma unroll
                for (int c = 0; c < 7; ++c) my[6 * N + c] = r[3 + c];
            }
            __syncthreads();
            const int m = min(PROXY_THREADS, e - c0);
            for (int j = 0; j < m; ++j) {
                const float* pj = sb + j * SBW;
                const float* q = pj + 6 * N;
#pragma unroll
                for (int r = 0; r < PER; ++r) {
                    const float lx = pj[ka[r]], ly = pj[N + kb[r]], lz = pj[2 * N + kc[r]];
                    const float lyz = ly * lz, L = lx * lyz;
                    const float gx = pj[3 * N + ka[r]] * lyz, gy = lx * pj[4 * N + kb[r]] * lz,
                                gz = lx * ly * pj[5 * N + kc[r]];
                    acc[r][0] += L * q[0];
                    acc[r][1] += gx * q[1] + gy * q[2] + gz * q[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) acc[r][2 + c] += L * q[4 + c];
#pragma unroll
                    for (int c = 0; c < 3; ++c) acc[r][5 + c] += L * q[1 + c];
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int k = threadIdx.x + r * PROXY_THREADS;
        if (k >= NP) break;
        float* o = prox + ((int64_t)slot * NP + k) * TREE_REC;
        o[0] = mid[0] + half[0] * tn[ka[r]];
        o[1] = mid[1] + half[1] * tn[kb[r]];
        o[2] = mid[2] + half[2] * tn[kc[r]];
#pragma unroll
        for (int c = 0; c < 8; ++c) o[3 + c] = acc[r][c];
        o[11] = 0.f;
    }
}

// Packed pairs of FP32 values (f32x2 instructions: two targets per thread).
// The treecode's own launch: one CTA per leaf of targets and split, TREE_LEAF
// threads in two groups (tree_leaf_body with NQ = 2); the linear block index
// walks the leaves longest first, a leaf's splits side by side.
template <int MODE>
__global__ void __launch_bounds__(TREE_LEAF, 7) k_tree_eval(TreeJob job) {
    __shared__ __align__(16) float tile[TREE_EVAL_TILE * (2 * TREE_REC + TREE_DUP)];
    static_assert((MODE == 0 ? 2 : 10) * TREE_LEAF <= TREE_EVAL_TILE * (2 * TREE_REC + TREE_DUP), "reduction buffer");
    const int sp = (int)(blockIdx.x % (unsigned)job.nsplit);
    tree_leaf_body<MODE, 2>(job, job.leaf_order[blockIdx.x / (unsigned)job.nsplit], sp, tile);
}

// y-part of the far field by the treecode: per-target partial sums in the
// direct kernel's split layout (*nsplit slices in the mesh's ws_part, returned
// in *part_out); builds the tree of the mesh on first use.
int tree_prepare(const pb_mesh* mc, const FarPlan& fp, const double* x, bool need_u, bool need_v, TreeJob* job,
                 cudaStream_t s) {
    pb_mesh* m = const_cast<pb_mesh*>(mc);
    pb_ctx* ctx = m->ctx;
    if (m->tree && (m->tree->n != ctx->tree_order + 1 || m->tree->theta != ctx->tree_theta)) {
        tree_free(m->tree);  // the settings changed: a new tree (captured graphs must not keep the old one)
        m->tree = nullptr;
        ++m->ws_gen;
    }
    if (!m->tree) PB_TRY(build_tree(m, ctx->tree_order, ctx->tree_theta, &m->tree));
    PbTree* t = m->tree;
    const int64_t np = m->np, nv = m->nv;
    PB_TRY(ws_reserve(m->ws_tree, sizeof(float) * TREE_REC * (np + (size_t)t->nslot * t->nprox) + 256));
    float* rec = (float*)m->ws_tree.ptr;
    float* prox = rec + TREE_REC * np;
    k_tree_sources<<<(unsigned)((np + 127) / 128), 128, 0, s>>>(np, m->Q, mesh_rule(m), t->perm, m->tris, m->tgeo,
                                                                m->pts64, m->pts32, x, x + nv, need_u, need_v, rec);
    ::pb::count_launch();
    for (size_t h = 0; h + 1 < t->height_ptr.size(); ++h) {  // children's proxies before their parents'
        const int64_t b = t->height_ptr[h], e = t->height_ptr[h + 1];
        if (e > b) {
            const unsigned g = (unsigned)(e - b);
            const int32_t* so = t->slot_order + b;
            switch (t->n) {
                case 3: k_proxy_charges<3><<<g, PROXY_THREADS, 0, s>>>(so, t->slot_kids, t->slot_box, rec, prox); break;
                case 4: k_proxy_charges<4><<<g, PROXY_THREADS, 0, s>>>(so, t->slot_kids, t->slot_box, rec, prox); break;
                case 5: k_proxy_charges<5><<<g, PROXY_THREADS, 0, s>>>(so, t->slot_kids, t->slot_box, rec, prox); break;
                case 6: k_proxy_charges<6><<<g, PROXY_THREADS, 0, s>>>(so, t->slot_kids, t->slot_box, rec, prox); break;
                case 7: k_proxy_charges<7><<<g, PROXY_THREADS, 0, s>>>(so, t->slot_kids, t->slot_box, rec, prox); break;
                default: k_proxy_charges<8><<<g, PROXY_THREADS, 0, s>>>(so, t->slot_kids, t->slot_box, rec, prox); break;
            }
            ::pb::count_launch();
        }
    }
    TreeJob& J = *job;
    for (int R = 0; R < 2; ++R)
        for (int j = 0; j < 4; ++j) J.cf.k[R][j] = (float)fp.k[R][j];
    J.cf.kappa = (float)fp.kappa;
    J.cf.mk2 = (float)(-fp.kappa * 1.4426950408889634);
    // splits of each leaf's lists, so that the grid holds about eight CTAs per SM
    const int nacc = fp.mode == 0 ? 2 : 10;
    const int S = (int)std::min<int64_t>(
        TREE_MAX_SPLITS, std::max<int64_t>(1, (8LL * std::max(1, ctx->num_sms) + t->nleaf - 1) / t->nleaf));
    PB_TRY(ws_reserve(m->ws_part, sizeof(float) * (size_t)S * nacc * np));
    J.np = np;
    J.nprox = t->nprox;
    J.nsplit = S;
    J.perm = t->perm;
    J.leaf_rng = t->leaf_rng;
    J.leaf_order = t->leaf_order;
    J.far_ptr = t->far_ptr;
    J.far_idx = t->far_idx;
    J.near_ptr = t->near_ptr;
    J.near_rng = t->near_rng;
    J.rec = rec;
    J.prox = prox;
    J.part = (float*)m->ws_part.ptr;
    PB_CUDA(cudaGetLastError());
    return PB_OK;
}

int64_t tree_interactions(const pb_mesh* m) { return m->tree ? m->tree->direct_pairs + m->tree->proxy_pairs : 0; }
int64_t tree_leaves(const pb_mesh* m) { return m->tree ? m->tree->nleaf : 0; }

int tree_far(const pb_mesh* m, const FarPlan& fp, const double* x, bool need_u, bool need_v, float** part_out,
             int* nsplit, cudaStream_t s) {
    TreeJob job;
    PB_TRY(tree_prepare(m, fp, x, need_u, need_v, &job, s));
    const PbTree* t = m->tree;
    const unsigned grid = (unsigned)(t->nleaf * job.nsplit);
    // FP32 operations per interaction as the evaluation does them (f32x2 lanes counted singly; the two
    // MUFU operations, rsqrt and ex2, not counted): a direct pair 24 (V/K rows) or 35 (V/K + D/T
    // rows), a proxy 12 or 29 (its charges come combined with the kernel coefficients)
    const double ops_near = fp.mode == 0 ? 24.0 : 35.0, ops_far = fp.mode == 0 ? 12.0 : 29.0;
    const double inter = (double)(t->direct_pairs + t->proxy_pairs);
    const double ops = ((double)t->direct_pairs * ops_near + (double)t->proxy_pairs * ops_far) / std::max(1.0, inter);
    Timer tm(m->ctx, PB_KERNEL_TREE32, s, inter, ops);
    if (fp.mode == 0) k_tree_eval<0><<<grid, TREE_LEAF, 0, s>>>(job);
    else k_tree_eval<1><<<grid, TREE_LEAF, 0, s>>>(job);
    ::pb::count_launch();
    tm.stop();
    PB_CUDA(cudaGetLastError());
    *part_out = job.part;
    *nsplit = job.nsplit;
    return PB_OK;
}

int tree_info(const pb_mesh* m, int64_t out[6]) {
    const PbTree* t = m->tree;
    if (!t) return set_error(PB_EINVAL, "pb_tree_info: the mesh has no tree (no treecode application yet)");
    out[0] = t->nleaf;
    out[1] = t->nslot;
    out[2] = t->n_far;
    out[3] = t->n_near;
    out[4] = t->direct_pairs;
    out[5] = t->proxy_pairs;
    return PB_OK;
}

}  // namespace pb
