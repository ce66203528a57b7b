// Treecode evaluation body (shared by the treecode's own launch and the
// request server's persistent launch). Not part of the C ABI.
#pragma once

#include "internal.h"

namespace pb {

constexpr int TREE_LEAF = 128;     // targets per leaf
constexpr int TREE_REC = 12;       // floats per tree source / proxy record in global memory
constexpr int TREE_DUP = 24;       // floats per record as summed from shared memory: every value twice,
                                   // so that one load gives both halves of a packed f32x2 operand
constexpr int TREE_EVAL_TILE = 128;  // sources staged per round

struct TreeCoef {
    float k[2][4];
    float kappa;
    float mk2;  // -kappa log2(e)
};

__device__ __forceinline__ float t_rsqrt(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float t_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 t_sub2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n sub.rn.f32x2 rd, ra, rb;\n"
        " mov.b64 {%0, %1}, rd;\n}\n" : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 t_mul2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mul.rn.f32x2 rd, ra, rb;\n"
        " mov.b64 {%0, %1}, rd;\n}\n" : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 t_fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
        " fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}\n"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 t_splat(float v) { return make_float2(v, v); }


// One evaluation job: a mesh's tree with its source and proxy records in
// tree order, the kernel coefficients and the partial-sum slices.
struct TreeJob {
    int64_t np;
    int nprox;
    int nsplit;                 // slices of partial sums (the leaves' lists are cut into nsplit shares)
    const int32_t* perm;        // tree index -> point index
    const int32_t* leaf_rng;    // 2 per leaf
    const int32_t* leaf_order;  // leaves by decreasing interaction count
    const int32_t* far_ptr;     // per leaf: its proxied clusters
    const int32_t* far_idx;
    const int32_t* near_ptr;    // per leaf: its directly summed source ranges
    const int32_t* near_rng;
    const float* rec;           // source records in tree order
    const float* prox;          // proxy records per slot
    float* part;                // nsplit x NACC x np
    TreeCoef cf;
};

// Asynchronous 16-byte copies global -> shared (cp.async), committed in groups:
// the staging of the next tile runs while the current one is summed.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// The tiles of one leaf's share of its lists, in order: every proxied cluster's
// proxies (far, in tiles of TREE_EVAL_TILE records), then every directly summed
// source range (near, likewise).
struct TreeTiles {
    int32_t f, fe, q, qe;  // list cursors
    int32_t off;           // records done in the current cluster or range
    __device__ __forceinline__ bool next(const TreeJob& T, const float** src, int* cnt, bool* far) {
        constexpr int TILE = TREE_EVAL_TILE;
        if (f < fe) {
            *src = T.prox + ((int64_t)T.far_idx[f] * T.nprox + off) * TREE_REC;
            *cnt = min(TILE, T.nprox - off);
            *far = true;
            off += TILE;
            if (off >= T.nprox) { ++f; off = 0; }
            return true;
        }
        while (q < qe) {
            const int32_t sb = T.near_rng[2 * q], se = T.near_rng[2 * q + 1];
            if (sb + off >= se) { ++q; off = 0; continue; }
            *src = T.rec + (int64_t)(sb + off) * TREE_REC;
            *cnt = min(TILE, se - sb - off);
            *far = false;
            off += TILE;
            if (sb + off >= se) { ++q; off = 0; }
            return true;
        }
        return false;
    }
};

// One leaf of targets and one split of its lists, on 64 NQ threads: a thread
// holds two targets (the leaf's i-th and (i + 64)-th points) in packed f32x2
// arithmetic; the NQ thread groups of 64 take every NQ-th source of each staged
// tile and add their sums through shared memory at the end, group 0 adding
// groups 1 .. NQ-1 in that order. Far: proxies of the well-separated clusters
// (kernel G with the interpolated charges). Near: the other sources directly,
// with the direct pair kernel's arithmetic (identical points skipped). Tiles
// are staged in two buffers by asynchronous copies, the next one in flight
// while the current one is summed; before it is summed a tile is copied once
// more inside shared memory with every value twice (TREE_DUP floats per
// record), which keeps the records in global memory (and L2) at 48 bytes, and
// with the charges that only meet constant kernel coefficients combined with
// them there (per record a, b with a + e b the Laplace + Yukawa weight, e =
// exp(-kappa r)), which takes 3 to 6 operations off every interaction.
// `tile` holds at least TREE_EVAL_TILE x (2 TREE_REC + TREE_DUP) floats and
// (NQ - 1) x NACC x TREE_LEAF floats. Every thread of the group calls it (it
// synchronises the CTA) and returns with no copy in flight.
template <int MODE, int NQ>
__device__ __forceinline__ void tree_leaf_body(const TreeJob& T, int leaf, int sp, float* tile) {
    constexpr int NACC = MODE == 0 ? 2 : 10;
    constexpr int TILE = TREE_EVAL_TILE;
    constexpr int HALF = TREE_LEAF / 2;
    constexpr int NTH = HALF * NQ;
    const int nsp = T.nsplit;
    const int32_t fb0 = T.far_ptr[leaf], nfar = T.far_ptr[leaf + 1] - fb0;
    const int32_t qb0 = T.near_ptr[leaf], nnear = T.near_ptr[leaf + 1] - qb0;
    const int32_t fb = fb0 + (int32_t)((int64_t)nfar * sp / nsp), fe = fb0 + (int32_t)((int64_t)nfar * (sp + 1) / nsp);
    const int32_t qb = qb0 + (int32_t)((int64_t)nnear * sp / nsp), qe = qb0 + (int32_t)((int64_t)nnear * (sp + 1) / nsp);
    const int64_t np = T.np;
    float* part = T.part + (int64_t)sp * NACC * np;
    const float* rec = T.rec;
    const int32_t tb = T.leaf_rng[2 * leaf], te = T.leaf_rng[2 * leaf + 1];
    const int grp = (int)threadIdx.x / HALF;
    const int32_t ti0 = tb + (int32_t)(threadIdx.x % HALF), ti1 = ti0 + HALF;
    const bool live0 = ti0 < te, live1 = ti1 < te;
    float2 X0 = t_splat(0.f), X1 = X0, X2 = X0;
    if (live0) {
        X0.x = rec[TREE_REC * (int64_t)ti0];
        X1.x = rec[TREE_REC * (int64_t)ti0 + 1];
        X2.x = rec[TREE_REC * (int64_t)ti0 + 2];
    }
    if (live1) {
        X0.y = rec[TREE_REC * (int64_t)ti1];
        X1.y = rec[TREE_REC * (int64_t)ti1 + 1];
        X2.y = rec[TREE_REC * (int64_t)ti1 + 2];
    }
    const TreeCoef& cf = T.cf;
    const float2 c00 = t_splat(cf.k[0][0]), c01 = t_splat(cf.k[0][1]), c02 = t_splat(cf.k[0][2]),
                 c03 = t_splat(cf.k[0][3]), c10 = t_splat(cf.k[1][0]), c11 = t_splat(cf.k[1][1]),
                 c12 = t_splat(cf.k[1][2]), c13 = t_splat(cf.k[1][3]), kap = t_splat(cf.kappa),
                 mk2 = t_splat(cf.mk2);
    float2 acc[NACC];
    for (int k = 0; k < NACC; ++k) acc[k] = t_splat(0.f);
    const bool any = live0;  // the first target of a thread is live whenever the second is
    TreeTiles it = {fb, fe, qb, qe, 0};
    const float* src = nullptr;
    int cnt = 0, cnt_next = 0;
    bool far = false, far_next = false;
    bool have = it.next(T, &src, &cnt, &far);
    __syncthreads();  // the buffers may still be read by the caller's previous work
    if (have) {
        for (int k = threadIdx.x; k < cnt * TREE_REC / 4; k += NTH) cp_async16(tile + 4 * k, src + 4 * k);
    }
    cp_async_commit();
    for (int buf = 0; have; buf ^= 1) {
        const float* nsrc = nullptr;
        const bool have_next = it.next(T, &nsrc, &cnt_next, &far_next);
        if (have_next) {
            float* nb = tile + (buf ^ 1) * TILE * TREE_REC;
            for (int k = threadIdx.x; k < cnt_next * TREE_REC / 4; k += NTH) cp_async16(nb + 4 * k, nsrc + 4 * k);
        }
        cp_async_commit();
        cp_async_wait<1>();  // this thread's copies of the current tile have landed
        __syncthreads();     // and every thread's; the duplicated tile's last readers are done
        float* dup = tile + 2 * TILE * TREE_REC;
        for (int r = threadIdx.x; r < cnt; r += NTH) {
            // a record as summed: the charges that only ever meet the kernel coefficients
            // combined with them once here (Laplace and Yukawa parts a + e b, e = exp(-kappa r))
            const float4* rp = reinterpret_cast<const float4*>(tile + buf * TILE * TREE_REC + TREE_REC * r);
            const float4 u0 = rp[0], u1 = rp[1], u2 = rp[2];
            float v[TREE_REC] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w, u2.x, u2.y, u2.z, u2.w};
            const float s_ = v[3];
            if (far) {
                const float q_ = v[4];  // proxy: x, S, Q, C, N
                if (MODE == 0) {        // x, (a, b) of both rows
                    v[3] = fmaf(cf.k[0][2], q_, cf.k[0][0] * s_);
                    v[4] = fmaf(cf.k[0][3], q_, cf.k[0][1] * s_);
                    v[5] = fmaf(cf.k[1][2], q_, cf.k[1][0] * s_);
                    v[6] = fmaf(cf.k[1][3], q_, cf.k[1][1] * s_);
                } else {  // x, S, (a, b) of the phi row, C, N
#pragma unroll
                    for (int k = TREE_REC - 1; k >= 6; --k) v[k] = v[k - 1];
                    v[4] = fmaf(cf.k[0][2], q_, cf.k[0][0] * s_);
                    v[5] = fmaf(cf.k[0][3], q_, cf.k[0][1] * s_);
                }
            } else if (MODE == 0) {  // source: x, s, p, (a, b) of both rows' single layers
                v[7] = cf.k[0][0] * s_;
                v[8] = cf.k[0][1] * s_;
                v[9] = cf.k[1][0] * s_;
                v[10] = cf.k[1][1] * s_;
            } else {  // x, s, p, c, (a, b) of the phi row's single layer
                v[10] = cf.k[0][0] * s_;
                v[11] = cf.k[0][1] * s_;
            }
            float4* d4 = reinterpret_cast<float4*>(dup + TREE_DUP * r);
#pragma unroll
            for (int h = 0; h < TREE_REC / 2; ++h) d4[h] = make_float4(v[2 * h], v[2 * h], v[2 * h + 1], v[2 * h + 1]);
        }
        __syncthreads();
        const float* cur = dup;
        if (any && far) {
#pragma unroll 2
            for (int j = grp; j < cnt; j += NQ) {
                // the record's values, each as a splatted pair
                const float4* z4 = reinterpret_cast<const float4*>(cur + TREE_DUP * j);
                const float4 a = z4[0], b = z4[1], c = z4[2];
                const float2 d0 = t_sub2(X0, make_float2(a.x, a.y)), d1 = t_sub2(X1, make_float2(a.z, a.w)),
                             d2 = t_sub2(X2, make_float2(b.x, b.y));
                const float2 r2 = t_fma2(d0, d0, t_fma2(d1, d1, t_mul2(d2, d2)));
                const float2 rinv = make_float2(t_rsqrt(r2.x), t_rsqrt(r2.y));
                const float2 rr = t_mul2(r2, rinv);
                const float2 arg = t_mul2(rr, mk2);
                const float2 e = make_float2(t_ex2(arg.x), t_ex2(arg.y));
                if (MODE == 0) {
                    const float4 dd = z4[3];
                    acc[0] = t_fma2(rinv, t_fma2(e, make_float2(c.x, c.y), make_float2(b.z, b.w)), acc[0]);
                    acc[1] = t_fma2(rinv, t_fma2(e, make_float2(dd.x, dd.y), make_float2(c.z, c.w)), acc[1]);
                } else {
                    acc[0] = t_fma2(rinv, t_fma2(e, make_float2(c.z, c.w), make_float2(c.x, c.y)), acc[0]);
                    const float2 ek = t_fma2(e, t_mul2(rr, kap), e);
                    const float2 ts = t_mul2(t_fma2(c13, ek, c12),
                                             t_mul2(t_mul2(rinv, rinv), t_mul2(rinv, make_float2(b.z, b.w))));
                    acc[1] = t_fma2(ts, d0, acc[1]);
                    acc[2] = t_fma2(ts, d1, acc[2]);
                    acc[3] = t_fma2(ts, d2, acc[3]);
                    const float4 dd = z4[3], ee = z4[4], ff = z4[5];
                    const float2 gc = t_mul2(t_fma2(c11, e, c10), rinv);
                    acc[4] = t_fma2(gc, make_float2(dd.x, dd.y), acc[4]);
                    acc[5] = t_fma2(gc, make_float2(dd.z, dd.w), acc[5]);
                    acc[6] = t_fma2(gc, make_float2(ee.x, ee.y), acc[6]);
                    const float2 gb = t_mul2(e, rinv);
                    acc[7] = t_fma2(gb, make_float2(ee.z, ee.w), acc[7]);
                    acc[8] = t_fma2(gb, make_float2(ff.x, ff.y), acc[8]);
                    acc[9] = t_fma2(gb, make_float2(ff.z, ff.w), acc[9]);
                }
            }
        } else if (any) {
#pragma unroll 2
            for (int j = grp; j < cnt; j += NQ) {
                const float4* y4 = reinterpret_cast<const float4*>(cur + TREE_DUP * j);
                const float4 a = y4[0], b = y4[1], c = y4[2], dd = y4[3], ee = y4[4], ff = y4[5];
                const float2 y3 = make_float2(b.z, b.w), p0 = make_float2(c.x, c.y), p1 = make_float2(c.z, c.w),
                             p2 = make_float2(dd.x, dd.y);
                const float2 d0 = t_sub2(X0, make_float2(a.x, a.y)), d1 = t_sub2(X1, make_float2(a.z, a.w)),
                             d2 = t_sub2(X2, make_float2(b.x, b.y));
                const float2 r2 = t_fma2(d0, d0, t_fma2(d1, d1, t_mul2(d2, d2)));
                const float2 rinv = make_float2(r2.x > 0.f ? t_rsqrt(r2.x) : 0.f, r2.y > 0.f ? t_rsqrt(r2.y) : 0.f);
                const float2 rr = t_mul2(r2, rinv);
                const float2 arg = t_mul2(rr, mk2);
                const float2 e = make_float2(t_ex2(arg.x), t_ex2(arg.y));
                const float2 ek = t_fma2(e, t_mul2(rr, kap), e);
                const float2 rinv3 = t_mul2(t_mul2(rinv, rinv), rinv);
                const float2 dp = t_fma2(d0, p0, t_fma2(d1, p1, t_mul2(d2, p2)));
                const float2 r3dp = t_mul2(rinv3, dp);
                if (MODE == 0) {
                    acc[0] = t_fma2(rinv, t_fma2(e, make_float2(ee.x, ee.y), make_float2(dd.z, dd.w)), acc[0]);
                    acc[0] = t_fma2(t_fma2(c03, ek, c02), r3dp, acc[0]);
                    acc[1] = t_fma2(rinv, t_fma2(e, make_float2(ff.x, ff.y), make_float2(ee.z, ee.w)), acc[1]);
                    acc[1] = t_fma2(t_fma2(c13, ek, c12), r3dp, acc[1]);
                } else {
                    acc[0] = t_fma2(rinv, t_fma2(e, make_float2(ff.z, ff.w), make_float2(ff.x, ff.y)), acc[0]);
                    acc[0] = t_fma2(t_fma2(c03, ek, c02), r3dp, acc[0]);
                    const float2 ts = t_mul2(t_fma2(c13, ek, c12), t_mul2(rinv3, y3));
                    acc[1] = t_fma2(ts, d0, acc[1]);
                    acc[2] = t_fma2(ts, d1, acc[2]);
                    acc[3] = t_fma2(ts, d2, acc[3]);
                    const float2 gc = t_mul2(t_fma2(c11, e, c10), rinv);
                    acc[4] = t_fma2(gc, make_float2(dd.z, dd.w), acc[4]);
                    acc[5] = t_fma2(gc, make_float2(ee.x, ee.y), acc[5]);
                    acc[6] = t_fma2(gc, make_float2(ee.z, ee.w), acc[6]);
                    const float2 gb = t_mul2(e, rinv);
                    acc[7] = t_fma2(gb, p0, acc[7]);
                    acc[8] = t_fma2(gb, p1, acc[8]);
                    acc[9] = t_fma2(gb, p2, acc[9]);
                }
            }
        }
        have = have_next;
        cnt = cnt_next;
        far = far_next;
    }
    cp_async_wait<0>();  // nothing in flight (the last group is empty)
    // the other groups' sums join group 0's, in group order
    __syncthreads();
    const int tl = (int)threadIdx.x % HALF;
    if (grp > 0) {
        float* slot = tile + (grp - 1) * NACC * TREE_LEAF;
        for (int k = 0; k < NACC; ++k) {
            slot[k * TREE_LEAF + tl] = acc[k].x;
            slot[k * TREE_LEAF + HALF + tl] = acc[k].y;
        }
    }
    __syncthreads();
    if (grp == 0) {
        for (int g2 = 1; g2 < NQ; ++g2) {
            const float* slot = tile + (g2 - 1) * NACC * TREE_LEAF;
            for (int k = 0; k < NACC; ++k) {
                acc[k].x += slot[k * TREE_LEAF + tl];
                acc[k].y += slot[k * TREE_LEAF + HALF + tl];
            }
        }
        if (live0) {
            const int64_t pt = T.perm[ti0];
            for (int k = 0; k < NACC; ++k) part[(int64_t)k * np + pt] = acc[k].x;
        }
        if (live1) {
            const int64_t pt = T.perm[ti1];
            for (int k = 0; k < NACC; ++k) part[(int64_t)k * np + pt] = acc[k].y;
        }
    }
    __syncthreads();  // the buffer is free for the caller
}

// host side (tree.cu): the mesh's tree built if needed, its source records and
// proxy charges computed on stream s for the far-field plan fp and the
// coefficients x, and the evaluation job described (partial sums in the mesh's
// ws_part, nsplit slices).
int tree_prepare(const pb_mesh* m, const FarPlan& fp, const double* x, bool need_u, bool need_v, TreeJob* job,
                 cudaStream_t s);
// pairs of one application (direct + proxy) and leaves, for cost estimates
int64_t tree_interactions(const pb_mesh* m);
int64_t tree_leaves(const pb_mesh* m);

}  // namespace pb
