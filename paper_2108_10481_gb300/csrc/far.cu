// a3 + a4 + a5: application of a 2x2 block operator y = B x.
//
//   far field  : every target quadrature point x_p against every source point
//                y_q (identical points skipped), Laplace and Yukawa fused:
//                G_L = 1/(4 pi r), G_Y = e^{-kappa r}/(4 pi r),
//                dG/dn_y = (x - y).n_y (1 + kappa r) e^{-kappa r}/(4 pi r^3)
//                (paper eq. layer_potentials with its Green's functions);
//   P1 maps    : coefficients -> source densities (a4 i), point sums -> test
//                functions by a gather over each vertex's triangles (a4 ii);
//   near field : the FP64 correction of pairs that share a vertex, as a
//                vertex-pair CSR SpMV fused with the gather (a5).
//
// Source record (12 slots): y(3), s = w v/(4 pi), p = w u n_y/(4 pi) (3),
// c = w curl u/(4 pi) (3), with w the point's rule weight times the area and
// curl u = sum_a u_a (-e_a / (2|tau|)) on the source triangle. The FP32
// record has 16 slots: the same 12 plus the low parts of y (split coordinates).
//
// Target accumulators of one kernel row:
//   phi-row (V, K):  sum rinv (cVL + cVY e) s + rinv^3 (cKL + cKY e (1+kappa r)) (d.p)
//   DT-row (D, T):   Tv = sum rinv^3 (cTL + cTY e(1+kappa r)) s d,   (T = -n_x.Tv)
//                    Cv = sum rinv (cDL + cDY e) c,                   (D curl part)
//                    Bv = sum rinv e p                               (D normal part x kappa^2 cDY)
// with d = x - y, e = exp(-kappa r).
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "internal.h"
#include "tree_eval.cuh"

namespace pb {

constexpr int REC64 = 12;  // doubles per FP64 source record
constexpr int REC32 = 16;  // floats per FP32 source record
constexpr double INV4PI = 0.07957747154594767;  // 1 / (4 pi)

// ------------------------------------------------------------ sources (a4 i)
template <typename T, int REC>
__global__ void k_sources(int64_t nt, int Q, Rule rule, const int32_t* __restrict__ tris,
                          const double* __restrict__ tgeo, const double* __restrict__ pts64,
                          const float* __restrict__ pts32, const float* __restrict__ pts32lo,
                          const double* __restrict__ u, const double* __restrict__ v, int need_u,
                          int need_v, T* __restrict__ rec) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double* g = tgeo + 16 * t;
    int32_t i0 = tris[3 * t], i1 = tris[3 * t + 1], i2 = tris[3 * t + 2];
    double ua[3] = {0, 0, 0}, va[3] = {0, 0, 0};
    if (need_u) { ua[0] = u[i0]; ua[1] = u[i1]; ua[2] = u[i2]; }
    if (need_v) { va[0] = v[i0]; va[1] = v[i1]; va[2] = v[i2]; }
    double inv2a = -1.0 / (2.0 * g[3]);
    double cu[3];
    for (int k = 0; k < 3; ++k) cu[k] = inv2a * (ua[0] * g[4 + k] + ua[1] * g[7 + k] + ua[2] * g[10 + k]);
    for (int q = 0; q < Q; ++q) {
        int64_t i = t * Q + q;
        double w = pts64[4 * i + 3] * INV4PI;
        double uq = rule.l[q][0] * ua[0] + rule.l[q][1] * ua[1] + rule.l[q][2] * ua[2];
        double vq = rule.l[q][0] * va[0] + rule.l[q][1] * va[1] + rule.l[q][2] * va[2];
        T* r = rec + REC * i;
        if (REC == REC64) {
            for (int k = 0; k < 3; ++k) r[k] = (T)pts64[4 * i + k];
        } else {
            for (int k = 0; k < 3; ++k) {
                r[k] = (T)pts32[4 * i + k];
                r[12 + k] = (T)pts32lo[4 * i + k];
            }
            r[15] = (T)0;
        }
        r[3] = (T)(w * vq);
        for (int k = 0; k < 3; ++k) {
            r[4 + k] = (T)(w * uq * g[k]);
            r[7 + k] = (T)(w * cu[k]);
        }
        if (REC == REC64) { r[10] = (T)0; r[11] = (T)0; }
        else { r[10] = (T)0; r[11] = (T)0; }
    }
}

// ------------------------------------------------------- FP64 pair kernel (a3)
constexpr int TPB64 = 128;  // threads (= targets) per CTA
constexpr int TS64 = 64;    // sources per shared-memory tile

struct Coef {
    double k[2][4];
    double kappa;
};

template <int MODE>
__global__ void __launch_bounds__(TPB64) k_pair64(int64_t np, const double* __restrict__ pts64,
                                                  const double* __restrict__ rec, Coef cf,
                                                  int64_t chunk, double* __restrict__ part) {
    constexpr int NACC = MODE == 0 ? 2 : 10;
    __shared__ double sh[TS64 * REC64];
    int64_t tgt = blockIdx.x * (int64_t)TPB64 + threadIdx.x;
    int split = blockIdx.y;
    int64_t j0 = split * chunk, j1 = min(np, j0 + chunk);
    bool live = tgt < np;
    double x0 = 0, x1 = 0, x2 = 0;
    if (live) { x0 = pts64[4 * tgt]; x1 = pts64[4 * tgt + 1]; x2 = pts64[4 * tgt + 2]; }
    double acc[NACC];
    for (int a = 0; a < NACC; ++a) acc[a] = 0.0;
    const double kap = cf.kappa;
    for (int64_t jt = j0; jt < j1; jt += TS64) {
        int nload = (int)min((int64_t)TS64, j1 - jt);
        for (int k = threadIdx.x; k < TS64 * REC64; k += TPB64)
            sh[k] = (k < nload * REC64) ? rec[jt * REC64 + k] : 0.0;
        __syncthreads();
        for (int j = 0; j < nload; ++j) {
            const double* s = sh + REC64 * j;
            double d0 = x0 - s[0], d1 = x1 - s[1], d2 = x2 - s[2];
            double r2 = d0 * d0 + d1 * d1 + d2 * d2;
            if (!(r2 > 0.0)) continue;  // identical point (coincident triangle)
            double rinv = 1.0 / sqrt(r2);
            double r = r2 * rinv;
            double e = exp(-kap * r);
            double ek = e * (1.0 + kap * r);
            double rinv3 = rinv * rinv * rinv;
            double dp = d0 * s[4] + d1 * s[5] + d2 * s[6];
            double rs = rinv * s[3], r3dp = rinv3 * dp;
            acc[0] += (cf.k[0][0] + cf.k[0][1] * e) * rs + (cf.k[0][2] + cf.k[0][3] * ek) * r3dp;
            if (MODE == 0) {
                acc[1] += (cf.k[1][0] + cf.k[1][1] * e) * rs + (cf.k[1][2] + cf.k[1][3] * ek) * r3dp;
            } else {
                double ts = (cf.k[1][2] + cf.k[1][3] * ek) * rinv3 * s[3];
                acc[1] += ts * d0; acc[2] += ts * d1; acc[3] += ts * d2;
                double gc = (cf.k[1][0] + cf.k[1][1] * e) * rinv;
                acc[4] += gc * s[7]; acc[5] += gc * s[8]; acc[6] += gc * s[9];
                double gb = e * rinv;
                acc[7] += gb * s[4]; acc[8] += gb * s[5]; acc[9] += gb * s[6];
            }
        }
        __syncthreads();
    }
    if (live)
        for (int a = 0; a < NACC; ++a) part[((int64_t)split * NACC + a) * np + tgt] = acc[a];
}

// ------------------------------------------------ FP32 pair kernel, TMA-fed (a3)
constexpr int TPB32 = 256;  // threads per CTA
constexpr int TGT32 = 2;    // targets per thread
constexpr int TS32 = 128;   // sources per TMA tile (box rows)
constexpr int ST32 = 3;     // pipeline stages

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
// bounded wait: gives up after ~2^22 polls and records the failure
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, int* status) {
    for (int i = 0; i < (1 << 22); ++i)
        if (mbar_try_wait(bar, phase)) return true;
    atomicExch(status, PB_ETIMEOUT);
    return false;
}
// The CTA acts on a wait's outcome as one: every thread polls the barrier
// (bounded), and the tile is used only if all of them saw it complete, so a
// wait that runs out in one thread sends every thread down the same exit path
// (no thread is left at a barrier the others never reach).
__device__ __forceinline__ bool cta_wait(uint64_t* bar, uint32_t phase, int* status) {
    return __syncthreads_and(mbar_wait(bar, phase, status) ? 1 : 0) != 0;
}
// Exit path after a failed wait at tile `it`: the copies still in flight are
// those of tiles it .. min(ntiles, it + stages) - 1, tile k on stage k % stages
// with phase parity (k / stages) & 1. One thread waits for each (bounded)
// before the CTA leaves, so no copy lands in shared memory after it is gone.
__device__ __forceinline__ void cta_drain(uint64_t* bar, int stages, int it, int ntiles) {
    if (threadIdx.x == 0)
        for (int k = it; k < ntiles && k < it + stages; ++k)
            for (int i = 0; i < (1 << 20); ++i)
                if (mbar_try_wait(&bar[k % stages], (uint32_t)((k / stages) & 1))) break;
    __syncthreads();
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct Coef32 {
    float k[2][4];
    float kappa;
    float mk2;  // -kappa * log2(e)
};

template <int MODE, bool ACC>
__global__ void __launch_bounds__(TPB32) k_pair32(const __grid_constant__ CUtensorMap tmap, int64_t np,
                                                  const float* __restrict__ pts32,
                                                  const float* __restrict__ pts32lo, Coef32 cf,
                                                  int64_t chunk, void* __restrict__ part_out,
                                                  int* __restrict__ status) {
    constexpr int NACC = MODE == 0 ? 2 : 10;
    __shared__ __align__(128) float sh[ST32][TS32 * REC32];
    __shared__ __align__(8) uint64_t bar[ST32];
    const int split = blockIdx.y;
    const int64_t j0 = split * chunk;
    const int64_t j1 = min(np, j0 + chunk);
    const int ntiles = (int)((j1 - j0 + TS32 - 1) / TS32);

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST32; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = 0; s < ST32 && s < ntiles; ++s) {
            mbar_expect_tx(&bar[s], TS32 * REC32 * sizeof(float));
            tma_load_2d(sh[s], &tmap, 0, (int)(j0 + (int64_t)s * TS32), &bar[s]);
        }
    }

    float x[TGT32][3], xl[TGT32][3];
    int64_t tg[TGT32];
    for (int t = 0; t < TGT32; ++t) {
        tg[t] = blockIdx.x * (int64_t)(TPB32 * TGT32) + t * TPB32 + threadIdx.x;
        int64_t i = tg[t] < np ? tg[t] : np - 1;
        for (int k = 0; k < 3; ++k) {
            x[t][k] = pts32[4 * i + k];
            xl[t][k] = ACC ? pts32lo[4 * i + k] : 0.0f;
        }
    }
    float acc[TGT32][NACC];
    double accd[TGT32][ACC ? NACC : 1];
    for (int t = 0; t < TGT32; ++t) {
        for (int a = 0; a < NACC; ++a) acc[t][a] = 0.0f;
        for (int a = 0; a < (ACC ? NACC : 1); ++a) accd[t][a] = 0.0;
    }
    const float kap = cf.kappa, mk2 = cf.mk2;
    int failed_at = -1;
    for (int it = 0; it < ntiles; ++it) {
        const int st = it % ST32;
        const uint32_t phase = (uint32_t)((it / ST32) & 1);
        if (!cta_wait(&bar[st], phase, status)) { failed_at = it; break; }
        const float* tile = sh[st];
#pragma unroll 2
        for (int j = 0; j < TS32; ++j) {
            const float4 s0 = *reinterpret_cast<const float4*>(tile + REC32 * j);
            const float4 s1 = *reinterpret_cast<const float4*>(tile + REC32 * j + 4);
            float4 s2 = make_float4(0.f, 0.f, 0.f, 0.f), s3 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (MODE == 1) s2 = *reinterpret_cast<const float4*>(tile + REC32 * j + 8);
            if (ACC) s3 = *reinterpret_cast<const float4*>(tile + REC32 * j + 12);
#pragma unroll
            for (int t = 0; t < TGT32; ++t) {
                float d0 = x[t][0] - s0.x, d1 = x[t][1] - s0.y, d2 = x[t][2] - s0.z;
                if (ACC) { d0 += xl[t][0] - s3.x; d1 += xl[t][1] - s3.y; d2 += xl[t][2] - s3.z; }
                float r2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
                float rinv = r2 > 0.0f ? rsqrt_approx(r2) : 0.0f;
                float r = r2 * rinv;
                float e = ex2_approx(r * mk2);
                float ek = fmaf(e, kap * r, e);
                float rinv3 = rinv * rinv * rinv;
                float dp = fmaf(d0, s1.x, fmaf(d1, s1.y, d2 * s1.z));
                float rs = rinv * s0.w, r3dp = rinv3 * dp;
                acc[t][0] = fmaf(fmaf(cf.k[0][1], e, cf.k[0][0]), rs, acc[t][0]);
                acc[t][0] = fmaf(fmaf(cf.k[0][3], ek, cf.k[0][2]), r3dp, acc[t][0]);
                if (MODE == 0) {
                    acc[t][1] = fmaf(fmaf(cf.k[1][1], e, cf.k[1][0]), rs, acc[t][1]);
                    acc[t][1] = fmaf(fmaf(cf.k[1][3], ek, cf.k[1][2]), r3dp, acc[t][1]);
                } else {
                    float ts = fmaf(cf.k[1][3], ek, cf.k[1][2]) * (rinv3 * s0.w);
                    acc[t][1] = fmaf(ts, d0, acc[t][1]);
                    acc[t][2] = fmaf(ts, d1, acc[t][2]);
                    acc[t][3] = fmaf(ts, d2, acc[t][3]);
                    float gc = fmaf(cf.k[1][1], e, cf.k[1][0]) * rinv;
                    acc[t][4] = fmaf(gc, s1.w, acc[t][4]);
                    acc[t][5] = fmaf(gc, s2.x, acc[t][5]);
                    acc[t][6] = fmaf(gc, s2.y, acc[t][6]);
                    float gb = e * rinv;
                    acc[t][7] = fmaf(gb, s1.x, acc[t][7]);
                    acc[t][8] = fmaf(gb, s1.y, acc[t][8]);
                    acc[t][9] = fmaf(gb, s1.z, acc[t][9]);
                }
            }
        }
        if (ACC) {
            for (int t = 0; t < TGT32; ++t)
                for (int a = 0; a < NACC; ++a) {
                    accd[t][a] += (double)acc[t][a];
                    acc[t][a] = 0.0f;
                }
        }
        __syncthreads();  // every thread is done with this stage
        if (threadIdx.x == 0 && it + ST32 < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&bar[st], TS32 * REC32 * sizeof(float));
            tma_load_2d(sh[st], &tmap, 0, (int)(j0 + (int64_t)(it + ST32) * TS32), &bar[st]);
        }
    }
    if (failed_at >= 0) {
        cta_drain(bar, ST32, failed_at, ntiles);
        return;
    }
    for (int t = 0; t < TGT32; ++t) {
        if (tg[t] >= np) continue;
        for (int a = 0; a < NACC; ++a) {
            int64_t o = ((int64_t)split * NACC + a) * np + tg[t];
            if (ACC) static_cast<double*>(part_out)[o] = accd[t][a];
            else static_cast<float*>(part_out)[o] = acc[t][a];
        }
    }
}

// ------------------------------------ FP32 pair kernel, packed f32x2 (a3)
// The same sums as k_pair32 with Blackwell's packed FP32 instructions: each
// thread holds its targets in pairs, so one fma/add/mul.rn.f32x2 advances two
// targets. Source values are stored twice in a 32-float record so that every
// packed operand is a register pair loaded straight from shared memory:
//   x x y y z z s s | px px py py pz pz cx cx | cy cy cz cz xl xl yl yl | zl zl - - - - - -
// The identical-point guard is needed only in tiles that overlap the CTA's
// own targets or run past the last point (zero-filled rows).
constexpr int REC2 = 32;   // floats per duplicated source record
constexpr int TPB2 = 256;  // threads per CTA
constexpr int TS2 = 64;    // records per TMA tile
constexpr int ST2 = 4;     // pipeline stages

__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n add.rn.f32x2 rd, ra, rb;\n"
        " mov.b64 {%0, %1}, rd;\n}\n" : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n sub.rn.f32x2 rd, ra, rb;\n"
        " mov.b64 {%0, %1}, rd;\n}\n" : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mul.rn.f32x2 rd, ra, rb;\n"
        " mov.b64 {%0, %1}, rd;\n}\n" : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
        " fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}\n"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 splat(float v) { return make_float2(v, v); }

template <typename T>
__global__ void k_sources2(int64_t nt, int Q, Rule rule, const int32_t* __restrict__ tris,
                           const double* __restrict__ tgeo, const double* __restrict__ pts64,
                           const float* __restrict__ pts32, const float* __restrict__ pts32lo,
                           const double* __restrict__ u, const double* __restrict__ v, int need_u, int need_v,
                           float* __restrict__ rec) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double* g = tgeo + 16 * t;
    int32_t i0 = tris[3 * t], i1 = tris[3 * t + 1], i2 = tris[3 * t + 2];
    double ua[3] = {0, 0, 0}, va[3] = {0, 0, 0};
    if (need_u) { ua[0] = u[i0]; ua[1] = u[i1]; ua[2] = u[i2]; }
    if (need_v) { va[0] = v[i0]; va[1] = v[i1]; va[2] = v[i2]; }
    double inv2a = -1.0 / (2.0 * g[3]);
    double cu[3];
    for (int k = 0; k < 3; ++k) cu[k] = inv2a * (ua[0] * g[4 + k] + ua[1] * g[7 + k] + ua[2] * g[10 + k]);
    for (int q = 0; q < Q; ++q) {
        int64_t i = t * Q + q;
        double w = pts64[4 * i + 3] * INV4PI;
        double uq = rule.l[q][0] * ua[0] + rule.l[q][1] * ua[1] + rule.l[q][2] * ua[2];
        double vq = rule.l[q][0] * va[0] + rule.l[q][1] * va[1] + rule.l[q][2] * va[2];
        float val[16] = {pts32[4 * i], pts32[4 * i + 1], pts32[4 * i + 2], (float)(w * vq),
                         (float)(w * uq * g[0]), (float)(w * uq * g[1]), (float)(w * uq * g[2]),
                         (float)(w * cu[0]), (float)(w * cu[1]), (float)(w * cu[2]),
                         pts32lo[4 * i], pts32lo[4 * i + 1], pts32lo[4 * i + 2], 0.f, 0.f, 0.f};
        float4* r = reinterpret_cast<float4*>(rec + REC2 * i);
        for (int k = 0; k < 8; ++k) r[k] = make_float4(val[2 * k], val[2 * k], val[2 * k + 1], val[2 * k + 1]);
    }
}

struct Coef2 {
    float2 c[2][4];
    float2 kap, mk2;
};

template <int MODE, bool ACC, int NPK, bool GUARD, int TS>
__device__ __forceinline__ void tile_x2(const float* __restrict__ tile, const float2 (&X)[NPK][3],
                                        const float2 (&XL)[NPK][3], float2 (&acc)[NPK][MODE == 0 ? 2 : 10],
                                        const Coef2& cf) {
#pragma unroll 2
    for (int j = 0; j < TS; ++j) {
        const float* r = tile + REC2 * j;
        const float4 q0 = *reinterpret_cast<const float4*>(r);
        const float4 q1 = *reinterpret_cast<const float4*>(r + 4);
        const float4 q2 = *reinterpret_cast<const float4*>(r + 8);
        const float4 q3 = *reinterpret_cast<const float4*>(r + 12);
        float4 q4 = make_float4(0.f, 0.f, 0.f, 0.f), q5 = q4, q6 = q4;
        if (MODE == 1) q4 = *reinterpret_cast<const float4*>(r + 16);
        if (ACC) {
            q5 = *reinterpret_cast<const float4*>(r + 20);
            q6 = *reinterpret_cast<const float4*>(r + 24);
        }
        const float2 Sx = make_float2(q0.x, q0.y), Sy = make_float2(q0.z, q0.w), Sz = make_float2(q1.x, q1.y);
        const float2 Ss = make_float2(q1.z, q1.w), Px = make_float2(q2.x, q2.y), Py = make_float2(q2.z, q2.w);
        const float2 Pz = make_float2(q3.x, q3.y);
#pragma unroll
        for (int p = 0; p < NPK; ++p) {
            float2 d0 = sub2(X[p][0], Sx), d1 = sub2(X[p][1], Sy), d2 = sub2(X[p][2], Sz);
            if (ACC) {
                d0 = add2(d0, sub2(XL[p][0], make_float2(q5.x, q5.y)));
                d1 = add2(d1, sub2(XL[p][1], make_float2(q5.z, q5.w)));
                d2 = add2(d2, sub2(XL[p][2], make_float2(q6.x, q6.y)));
            }
            const float2 r2 = fma2(d0, d0, fma2(d1, d1, mul2(d2, d2)));
            float2 rinv = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
            if (GUARD) {
                rinv.x = r2.x > 0.0f ? rinv.x : 0.0f;
                rinv.y = r2.y > 0.0f ? rinv.y : 0.0f;
            }
            const float2 rr = mul2(r2, rinv);
            const float2 arg = mul2(rr, cf.mk2);
            const float2 e = make_float2(ex2_approx(arg.x), ex2_approx(arg.y));
            const float2 ek = fma2(e, mul2(rr, cf.kap), e);
            const float2 rinv3 = mul2(mul2(rinv, rinv), rinv);
            const float2 dp = fma2(d0, Px, fma2(d1, Py, mul2(d2, Pz)));
            const float2 rs = mul2(rinv, Ss), r3dp = mul2(rinv3, dp);
            acc[p][0] = fma2(fma2(cf.c[0][1], e, cf.c[0][0]), rs, acc[p][0]);
            acc[p][0] = fma2(fma2(cf.c[0][3], ek, cf.c[0][2]), r3dp, acc[p][0]);
            if (MODE == 0) {
                acc[p][1] = fma2(fma2(cf.c[1][1], e, cf.c[1][0]), rs, acc[p][1]);
                acc[p][1] = fma2(fma2(cf.c[1][3], ek, cf.c[1][2]), r3dp, acc[p][1]);
            } else {
                const float2 ts = mul2(fma2(cf.c[1][3], ek, cf.c[1][2]), mul2(rinv3, Ss));
                acc[p][1] = fma2(ts, d0, acc[p][1]);
                acc[p][2] = fma2(ts, d1, acc[p][2]);
                acc[p][3] = fma2(ts, d2, acc[p][3]);
                const float2 gc = mul2(fma2(cf.c[1][1], e, cf.c[1][0]), rinv);
                acc[p][4] = fma2(gc, make_float2(q3.z, q3.w), acc[p][4]);
                acc[p][5] = fma2(gc, make_float2(q4.x, q4.y), acc[p][5]);
                acc[p][6] = fma2(gc, make_float2(q4.z, q4.w), acc[p][6]);
                const float2 gb = mul2(e, rinv);
                acc[p][7] = fma2(gb, Px, acc[p][7]);
                acc[p][8] = fma2(gb, Py, acc[p][8]);
                acc[p][9] = fma2(gb, Pz, acc[p][9]);
            }
        }
    }
}

// Templated on its launch shape: source records per TMA tile (TS), pipeline
// stages (ST), packed target pairs per thread (NPK) and, for the
// split-coordinate variant, the tiles whose FP32 sums are added into the FP64
// sums at a time (PROMO: each FP64 addition takes about as much of the GB300's
// FP64 pipe as 64 FP32 operations take of the FMA pipe); the autotuner picks
// the shape per mesh-size bucket.
template <int MODE, bool ACC, int TS, int ST, int NPK, int PROMO = 1>
__global__ void __launch_bounds__(TPB2) k_pair32x2(const __grid_constant__ CUtensorMap tmap, int64_t np,
                                                   const float* __restrict__ pts32, const float* __restrict__ pts32lo,
                                                   Coef32 c32, int64_t chunk, void* __restrict__ part_out,
                                                   int* __restrict__ status) {
    constexpr int NACC = MODE == 0 ? 2 : 10;
    constexpr int TGT = 2 * NPK;
    __shared__ __align__(128) float sh[ST][TS * REC2];
    __shared__ __align__(8) uint64_t bar[ST];
    const int split = blockIdx.y;
    const int64_t j0 = split * chunk;
    const int64_t j1 = min(np, j0 + chunk);
    const int ntiles = (int)((j1 - j0 + TS - 1) / TS);
    const int64_t blk0 = blockIdx.x * (int64_t)(TPB2 * TGT), blk1 = blk0 + TPB2 * TGT;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = 0; s < ST && s < ntiles; ++s) {
            mbar_expect_tx(&bar[s], TS * REC2 * sizeof(float));
            tma_load_2d(sh[s], &tmap, 0, (int)(j0 + (int64_t)s * TS), &bar[s]);
        }
    }
    Coef2 cf;
    for (int R = 0; R < 2; ++R)
        for (int k = 0; k < 4; ++k) cf.c[R][k] = splat(c32.k[R][k]);
    cf.kap = splat(c32.kappa);
    cf.mk2 = splat(c32.mk2);
    float2 X[NPK][3], XL[NPK][3];
    int64_t tg[TGT];
    for (int t = 0; t < TGT; ++t) tg[t] = blk0 + t * TPB2 + threadIdx.x;
    for (int p = 0; p < NPK; ++p) {
        int64_t a = tg[2 * p] < np ? tg[2 * p] : np - 1;
        int64_t b = tg[2 * p + 1] < np ? tg[2 * p + 1] : np - 1;
        for (int k = 0; k < 3; ++k) {
            X[p][k] = make_float2(pts32[4 * a + k], pts32[4 * b + k]);
            XL[p][k] = ACC ? make_float2(pts32lo[4 * a + k], pts32lo[4 * b + k]) : make_float2(0.f, 0.f);
        }
    }
    float2 acc[NPK][NACC];
    double accd[TGT][ACC ? NACC : 1];
    for (int p = 0; p < NPK; ++p)
        for (int a = 0; a < NACC; ++a) acc[p][a] = make_float2(0.f, 0.f);
    for (int t = 0; t < TGT; ++t)
        for (int a = 0; a < (ACC ? NACC : 1); ++a) accd[t][a] = 0.0;
    int failed_at = -1;
    for (int it = 0; it < ntiles; ++it) {
        const int st = it % ST;
        const uint32_t phase = (uint32_t)((it / ST) & 1);
        if (!cta_wait(&bar[st], phase, status)) { failed_at = it; break; }
        const int64_t jt = j0 + (int64_t)it * TS;
        const bool guard = (jt < blk1 && jt + TS > blk0) || jt + TS > np;
        if (guard) tile_x2<MODE, ACC, NPK, true, TS>(sh[st], X, XL, acc, cf);
        else tile_x2<MODE, ACC, NPK, false, TS>(sh[st], X, XL, acc, cf);
        if (ACC && ((it + 1) % PROMO == 0 || it + 1 == ntiles)) {
            for (int p = 0; p < NPK; ++p)
                for (int a = 0; a < NACC; ++a) {
                    accd[2 * p][a] += (double)acc[p][a].x;
                    accd[2 * p + 1][a] += (double)acc[p][a].y;
                    acc[p][a] = make_float2(0.f, 0.f);
                }
        }
        __syncthreads();  // every thread is done with this stage
        if (threadIdx.x == 0 && it + ST < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&bar[st], TS * REC2 * sizeof(float));
            tma_load_2d(sh[st], &tmap, 0, (int)(j0 + (int64_t)(it + ST) * TS), &bar[st]);
        }
    }
    if (failed_at >= 0) {
        cta_drain(bar, ST, failed_at, ntiles);
        return;
    }
    for (int t = 0; t < TGT; ++t) {
        if (tg[t] >= np) continue;
        const int p = t >> 1, h = t & 1;
        for (int a = 0; a < NACC; ++a) {
            int64_t o = ((int64_t)split * NACC + a) * np + tg[t];
            if (ACC) static_cast<double*>(part_out)[o] = accd[t][a];
            else static_cast<float*>(part_out)[o] = h ? acc[p][a].y : acc[p][a].x;
        }
    }
}

// Launch shapes of the packed kernel, one table per row mode and variant; the
// autotuner picks one per mesh-size bucket (shape 0: the default).
// Shapes: (records per tile, stages, packed target pairs per thread, tiles per
// FP64 addition of the split-coordinate variant).
typedef void (*X2Launch)(dim3, cudaStream_t, const CUtensorMap&, int64_t, const float*, const float*, Coef32,
                         int64_t, void*, int*);
struct X2Entry {
    int ts, st, npk, promo;
    const void* fn;
    X2Launch launch;
};
constexpr int X2_SHAPES = 4;

template <int MODE, bool ACC, int TS, int ST, int NPK, int PROMO>
static void x2_launch(dim3 g, cudaStream_t s, const CUtensorMap& map, int64_t np, const float* p32,
                      const float* plo, Coef32 cf, int64_t chunk, void* part, int* status) {
    k_pair32x2<MODE, ACC, TS, ST, NPK, PROMO><<<g, TPB2, 0, s>>>(map, np, p32, plo, cf, chunk, part, status);
}
template <int MODE, bool ACC, int TS, int ST, int NPK, int PROMO = 1>
static X2Entry x2_entry() {
    return {TS, ST, NPK, PROMO, (const void*)k_pair32x2<MODE, ACC, TS, ST, NPK, PROMO>,
            x2_launch<MODE, ACC, TS, ST, NPK, PROMO>};
}
template <int MODE>
static void x2_row(X2Entry (&fast)[X2_SHAPES], X2Entry (&acc)[X2_SHAPES]) {
    fast[0] = x2_entry<MODE, false, 64, 4, 2>();
    fast[1] = x2_entry<MODE, false, 32, 4, 2>();
    fast[2] = x2_entry<MODE, false, 128, 2, 2>();
    fast[3] = x2_entry<MODE, false, 64, 4, 1>();
    acc[0] = x2_entry<MODE, true, 64, 4, 1>();
    acc[1] = x2_entry<MODE, true, 128, 2, 1>();
    acc[2] = x2_entry<MODE, true, 128, 2, 1, 2>();
    acc[3] = x2_entry<MODE, true, 64, 4, 1, 4>();
}
static const X2Entry& x2_kernel(int mode, bool acc, int shape) {
    struct Table {
        X2Entry e[2][2][X2_SHAPES];
        Table() {
            x2_row<0>(e[0][0], e[0][1]);
            x2_row<1>(e[1][0], e[1][1]);
        }
    };
    static const Table t;
    return t.e[mode ? 1 : 0][acc ? 1 : 0][(shape >= 0 && shape < X2_SHAPES) ? shape : 0];
}

// ------------------------- batched FP32 pair kernel: many meshes in one launch
// Work item = (job, target block, source split); the per-job split count and
// chunk are the ones the single-mesh path chooses, so every job's partial sums
// are bit-identical to a launch for that mesh alone. Source tiles are staged
// with plain bulk copies (no tensor map per job); every job's record array is
// padded with zero records to whole tiles.
struct PairJob {
    const float* rec;
    const float* pts32;
    const float* pts32lo;
    void* part;
    int64_t np;
    int64_t chunk;
    Coef32 cf;
    int nsplit;
    int pad;
};
struct PairItem {
    int job;    // index into the pair jobs (kind 0) or the tree jobs (kind 1)
    int tb;     // target block (kind 0) or leaf (kind 1)
    int split;  // source split (kind 0) or split of the leaf's lists (kind 1)
    int kind;
};

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Persistent form: a grid of at most one wave of CTAs (the SM count times the
// resident CTAs per SM) that take work items from the table in order through
// a global counter until it runs out; the host lists the items most expensive
// first, so that the last wave is made of short items. An item's sums do not
// depend on which CTA takes it. Two kinds of item share the table: a target
// block and source split of a direct pair sum (kind 0), and a leaf and list
// split of a treecode evaluation (kind 1, FP32 only: tree_leaf_body on the
// CTA's 256 threads, four groups of 64 over the sources, the staging buffer
// as its scratch). The staging pipeline of the pair items runs on across
// items: g counts the tiles a CTA has consumed, so tile it of the current item
// sits on stage (g + it) % ST2 with phase parity ((g + it) / ST2) & 1.
template <int MODE, bool ACC>
__global__ void __launch_bounds__(TPB2) k_pair32x2_queue(const PairJob* __restrict__ jobs,
                                                         const TreeJob* __restrict__ tjobs,
                                                         const PairItem* __restrict__ items, int n_items,
                                                         int* __restrict__ counter, int* __restrict__ status) {
    constexpr int NACC = MODE == 0 ? 2 : 10;
    constexpr int NPK = ACC ? 1 : 2;
    constexpr int TGT = 2 * NPK;
    __shared__ __align__(128) float sh[ST2][TS2 * REC2];
    __shared__ __align__(8) uint64_t bar[ST2];
    __shared__ int s_item;
    const uint32_t tile_bytes = TS2 * REC2 * sizeof(float);
    if (threadIdx.x == 0) {
        for (int st = 0; st < ST2; ++st) mbar_init(&bar[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t g = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();  // every thread has read s_item before it is written again
        if (item >= n_items) break;
        const PairItem it0 = items[item];
        if (it0.kind == 1) {
            if (!ACC) {
                static_assert(ST2 * TS2 * REC2 >= TREE_EVAL_TILE * (2 * TREE_REC + TREE_DUP) &&
                              ST2 * TS2 * REC2 >= 3 * (MODE == 0 ? 2 : 10) * TREE_LEAF, "tree scratch");
                static_assert(TPB2 == 4 * (TREE_LEAF / 2), "tree groups");
                tree_leaf_body<MODE, 4>(tjobs[it0.job], it0.tb, it0.split, &sh[0][0]);
            }
            continue;
        }
        const PairJob& J = jobs[it0.job];
        const int64_t np = J.np;
        const int split = it0.split;
        const int64_t j0 = split * J.chunk;
        const int64_t j1 = min(np, j0 + J.chunk);
        const int ntiles = (int)((j1 - j0 + TS2 - 1) / TS2);
        const int64_t blk0 = (int64_t)it0.tb * (TPB2 * TGT), blk1 = blk0 + TPB2 * TGT;
        if (threadIdx.x == 0) {
            // the stages were last read through the generic proxy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int k = 0; k < ST2 && k < ntiles; ++k) {
                const int st = (int)((g + k) % ST2);
                mbar_expect_tx(&bar[st], tile_bytes);
                bulk_load(sh[st], J.rec + (j0 + (int64_t)k * TS2) * REC2, tile_bytes, &bar[st]);
            }
        }
        Coef2 cf;
        for (int R = 0; R < 2; ++R)
            for (int k = 0; k < 4; ++k) cf.c[R][k] = splat(J.cf.k[R][k]);
        cf.kap = splat(J.cf.kappa);
        cf.mk2 = splat(J.cf.mk2);
        float2 X[NPK][3], XL[NPK][3];
        int64_t tg[TGT];
        for (int t = 0; t < TGT; ++t) tg[t] = blk0 + t * TPB2 + threadIdx.x;
        for (int p = 0; p < NPK; ++p) {
            int64_t a = tg[2 * p] < np ? tg[2 * p] : np - 1;
            int64_t b = tg[2 * p + 1] < np ? tg[2 * p + 1] : np - 1;
            for (int k = 0; k < 3; ++k) {
                X[p][k] = make_float2(J.pts32[4 * a + k], J.pts32[4 * b + k]);
                XL[p][k] = ACC ? make_float2(J.pts32lo[4 * a + k], J.pts32lo[4 * b + k]) : make_float2(0.f, 0.f);
            }
        }
        float2 acc[NPK][NACC];
        double accd[TGT][ACC ? NACC : 1];
        for (int p = 0; p < NPK; ++p)
            for (int a = 0; a < NACC; ++a) acc[p][a] = make_float2(0.f, 0.f);
        for (int t = 0; t < TGT; ++t)
            for (int a = 0; a < (ACC ? NACC : 1); ++a) accd[t][a] = 0.0;
        int failed_at = -1;
        for (int it = 0; it < ntiles; ++it) {
            const int st = (int)((g + it) % ST2);
            const uint32_t phase = (uint32_t)(((g + it) / ST2) & 1);
            if (!cta_wait(&bar[st], phase, status)) { failed_at = it; break; }
            const int64_t jt = j0 + (int64_t)it * TS2;
            const bool guard = (jt < blk1 && jt + TS2 > blk0) || jt + TS2 > np;
            if (guard) tile_x2<MODE, ACC, NPK, true, TS2>(sh[st], X, XL, acc, cf);
            else tile_x2<MODE, ACC, NPK, false, TS2>(sh[st], X, XL, acc, cf);
            if (ACC) {
                for (int p = 0; p < NPK; ++p)
                    for (int a = 0; a < NACC; ++a) {
                        accd[2 * p][a] += (double)acc[p][a].x;
                        accd[2 * p + 1][a] += (double)acc[p][a].y;
                        acc[p][a] = make_float2(0.f, 0.f);
                    }
            }
            __syncthreads();
            if (threadIdx.x == 0 && it + ST2 < ntiles) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&bar[st], tile_bytes);
                bulk_load(sh[st], J.rec + (j0 + (int64_t)(it + ST2) * TS2) * REC2, tile_bytes, &bar[st]);
            }
        }
        if (failed_at >= 0) {
            // the copies still in flight (tiles failed_at .. failed_at + ST2 - 1), then leave
            if (threadIdx.x == 0)
                for (int k = failed_at; k < ntiles && k < failed_at + ST2; ++k)
                    for (int i = 0; i < (1 << 20); ++i)
                        if (mbar_try_wait(&bar[(g + k) % ST2], (uint32_t)(((g + k) / ST2) & 1))) break;
            __syncthreads();
            return;
        }
        for (int t = 0; t < TGT; ++t) {
            if (tg[t] >= np) continue;
            const int p = t >> 1, h = t & 1;
            for (int a = 0; a < NACC; ++a) {
                int64_t o = ((int64_t)split * NACC + a) * np + tg[t];
                if (ACC) static_cast<double*>(J.part)[o] = accd[t][a];
                else static_cast<float*>(J.part)[o] = h ? acc[p][a].y : acc[p][a].x;
            }
        }
        g += (uint32_t)ntiles;
    }
}

// --------------------------------------------- point sums -> test functions (a4 ii)
template <typename P>
__global__ void k_tri_reduce(int64_t nt, int64_t np, Rule rule, int nsplit, int mode, FarPlan fp,
                             const double* __restrict__ tgeo, const double* __restrict__ pts64,
                             const P* __restrict__ part, double* __restrict__ tri_out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int Q = rule.Q;
    const int NACC = mode == 0 ? 2 : 10;
    const double* g = tgeo + 16 * t;
    double out[2][3] = {{0, 0, 0}, {0, 0, 0}};
    double ctot[3] = {0, 0, 0};
    for (int q = 0; q < Q; ++q) {
        int64_t i = t * Q + q;
        double w = pts64[4 * i + 3];
        double a[10];
        for (int k = 0; k < NACC; ++k) {
            double s = 0.0;
            for (int sp = 0; sp < nsplit; ++sp) s += (double)part[((int64_t)sp * NACC + k) * np + i];
            a[k] = s;
        }
        // kernel row 0: phi-row
        for (int b = 0; b < 3; ++b) out[0][b] += w * rule.l[q][b] * a[0];
        if (mode == 0) {
            for (int b = 0; b < 3; ++b) out[1][b] += w * rule.l[q][b] * a[1];
        } else {
            double nT = g[0] * a[1] + g[1] * a[2] + g[2] * a[3];
            double nB = g[0] * a[7] + g[1] * a[8] + g[2] * a[9];
            double sc = -nT + fp.kappa * fp.kappa * fp.k[1][1] * nB;
            for (int b = 0; b < 3; ++b) out[1][b] += w * rule.l[q][b] * sc;
            for (int k = 0; k < 3; ++k) ctot[k] += w * a[4 + k];
        }
    }
    if (mode == 1) {
        double inv2a = -1.0 / (2.0 * g[3]);
        for (int b = 0; b < 3; ++b) {
            const double* e = g + 4 + 3 * b;
            out[1][b] += inv2a * (e[0] * ctot[0] + e[1] * ctot[1] + e[2] * ctot[2]);
        }
    }
    double* o = tri_out + 6 * t;
    for (int r = 0; r < 2; ++r)
        for (int b = 0; b < 3; ++b) o[3 * fp.out_row[r] + b] = out[r][b];
}

// ------------------------------------- gather + near-field SpMV (a4 ii + a5)
// 8 lanes per vertex; lane-strided sums reduced by shuffles in a fixed order.
// The four combined block values of an entry lie together (comb[4 k + 2 r + c]),
// so one vector load (float4, or two double2) brings them.
template <typename V>
__global__ void k_gather_spmv(int64_t nv, const int32_t* __restrict__ v2t_ptr, const int32_t* __restrict__ v2t,
                              const double* __restrict__ tri, int use_far, const int32_t* __restrict__ row_ptr,
                              const int32_t* __restrict__ col, const V* __restrict__ comb, int64_t nnz,
                              const double* __restrict__ x, double* __restrict__ y) {
    int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t i = gid >> 3;
    int lane = threadIdx.x & 7;
    double y0 = 0.0, y1 = 0.0;
    if (i < nv) {
        if (use_far)
            for (int32_t k = v2t_ptr[i] + lane; k < v2t_ptr[i + 1]; k += 8) {
                int32_t ta = v2t[k];
                int64_t t = ta / 3;
                int a = ta - 3 * (int)t;
                y0 += tri[6 * t + a];
                y1 += tri[6 * t + 3 + a];
            }
        const double* u = x;
        const double* v = x + nv;
        for (int32_t k = row_ptr[i] + lane; k < row_ptr[i + 1]; k += 8) {
            const int32_t c = col[k];
            const double uc = u[c], vc = v[c];
            double b0, b1, b2, b3;
            if (sizeof(V) == 4) {
                const float4 f = reinterpret_cast<const float4*>(comb)[k];
                b0 = f.x; b1 = f.y; b2 = f.z; b3 = f.w;
            } else {
                const double2 lo = reinterpret_cast<const double2*>(comb)[2 * k];
                const double2 hi = reinterpret_cast<const double2*>(comb)[2 * k + 1];
                b0 = lo.x; b1 = lo.y; b2 = hi.x; b3 = hi.y;
            }
            y0 += b0 * uc + b1 * vc;
            y1 += b2 * uc + b3 * vc;
        }
    }
    for (int o = 4; o > 0; o >>= 1) {
        y0 += __shfl_xor_sync(0xffffffffu, y0, o, 8);
        y1 += __shfl_xor_sync(0xffffffffu, y1, o, 8);
    }
    if (i < nv && lane == 0) {
        y[i] = y0;
        y[nv + i] = y1;
    }
}

// ------------------------------------------------------------ near combine
__global__ void k_combine(int64_t nnz, const double* __restrict__ val, const int32_t* __restrict__ tpos,
                          BlockOp B, double* __restrict__ c64, float* __restrict__ c32) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    int64_t et = tpos[e];
    double vals[O_N];
    vals[O_M] = val[N_M * nnz + e];
    vals[O_VL] = val[N_VL * nnz + e];
    vals[O_KL] = val[N_KL * nnz + e];
    vals[O_TL] = val[N_KL * nnz + et];
    vals[O_DL] = val[N_DL * nnz + e];
    vals[O_VY] = val[N_VY * nnz + e];
    vals[O_KY] = val[N_KY * nnz + e];
    vals[O_TY] = val[N_KY * nnz + et];
    vals[O_DY] = val[N_DY * nnz + e];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double s = 0.0;
            for (int o = 0; o < O_N; ++o) s += B.c[r][c][o] * vals[o];
            c64[4 * e + 2 * r + c] = s;
            c32[4 * e + 2 * r + c] = (float)s;
        }
}

int combine_near(const pb_mesh* m, const pb_near* nf, const BlockOp& B, double* c64, float* c32,
                 cudaStream_t s) {
    k_combine<<<(unsigned)((m->nnz + 255) / 256), 256, 0, s>>>(m->nnz, nf->val, m->tpos, B, c64, c32); ::pb::count_launch();
    PB_CUDA(cudaGetLastError());
    return PB_OK;
}

// ------------------------------------------------------------- far plan
int make_far_plan(const BlockOp& B, double kappa, FarPlan* fp) {
    int kind[2];  // 0: phi-row, 1: DT-row
    double k[2][4];
    for (int R = 0; R < 2; ++R) {
        const double* cu = B.c[R][0];
        const double* cv = B.c[R][1];
        if (cu[O_VL] != 0 || cu[O_VY] != 0 || cu[O_TL] != 0 || cu[O_TY] != 0 || cv[O_KL] != 0 ||
            cv[O_KY] != 0 || cv[O_DL] != 0 || cv[O_DY] != 0)
            return set_error(PB_EINVAL, "block operator acts with V/T on u or K/D on v");
        bool phi = cv[O_VL] != 0 || cv[O_VY] != 0 || cu[O_KL] != 0 || cu[O_KY] != 0;
        bool dt = cu[O_DL] != 0 || cu[O_DY] != 0 || cv[O_TL] != 0 || cv[O_TY] != 0;
        if (phi && dt) return set_error(PB_EINVAL, "a block row mixes V/K with D/T terms");
        kind[R] = dt ? 1 : 0;
        if (dt) { k[R][0] = cu[O_DL]; k[R][1] = cu[O_DY]; k[R][2] = cv[O_TL]; k[R][3] = cv[O_TY]; }
        else { k[R][0] = cv[O_VL]; k[R][1] = cv[O_VY]; k[R][2] = cu[O_KL]; k[R][3] = cu[O_KY]; }
    }
    if (kind[0] == 1 && kind[1] == 1) return set_error(PB_EINVAL, "two D/T rows are not supported");
    fp->kappa = kappa;
    fp->any = false;
    for (int R = 0; R < 2; ++R)
        for (int j = 0; j < 4; ++j) fp->any = fp->any || k[R][j] != 0.0;
    if (kind[0] == 0 && kind[1] == 0) {
        fp->mode = 0;
        fp->out_row[0] = 0;
        fp->out_row[1] = 1;
        for (int j = 0; j < 4; ++j) { fp->k[0][j] = k[0][j]; fp->k[1][j] = k[1][j]; }
    } else {
        int rphi = kind[0] == 0 ? 0 : 1, rdt = 1 - rphi;
        fp->mode = 1;
        fp->out_row[0] = rphi;
        fp->out_row[1] = rdt;
        for (int j = 0; j < 4; ++j) { fp->k[0][j] = k[rphi][j]; fp->k[1][j] = k[rdt][j]; }
    }
    return PB_OK;
}

// split count: fill the GPU in whole waves (see the layout notes in the design)
static int choose_splits(int64_t np, int tpc, int tile, int slots) {
    int64_t nb = (np + tpc - 1) / tpc;
    int64_t ntiles = (np + tile - 1) / tile;
    int best = 1;
    double best_cost = 1e300;
    for (int S = 1; S <= 32; ++S) {
        if (S > ntiles) break;
        int64_t ctas = nb * S;
        int64_t waves = (ctas + slots - 1) / slots;
        int64_t per = (ntiles + S - 1) / S;
        double cost = (double)waves * (double)per * (1.0 + 0.01 * S);
        if (cost < best_cost) { best_cost = cost; best = S; }
    }
    return best;
}

int tune_bucket(int64_t np) {
    int b = 0;
    while (b + 1 < TUNE_BUCKETS && ((int64_t)1 << (b + 1)) <= np) ++b;
    return b;
}

TuneEntry tuned(const pb_ctx* ctx, int64_t np, int mode, bool acc) {
    return ctx->tune[mode ? 1 : 0][acc ? 1 : 0][tune_bucket(np)];
}

// split count after the tuned scale, within [1, tiles] and <= 32
static int scaled_splits(int S, double scale, int64_t np, int tile) {
    const int64_t ntiles = (np + tile - 1) / tile;
    int s2 = (int)(S * scale + 0.5);
    s2 = std::max(1, std::min(s2, 32));
    return (int)std::min<int64_t>(s2, ntiles);
}

static int occupancy_slots(const pb_mesh* m, const void* kern, int threads) {
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    cudaGetLastError();
    return per_sm * m->ctx->num_sms;
}

static int make_tmap(const pb_mesh* m, const float* rec, CUtensorMap* map, int rec_floats = REC32,
                     int box_rows = TS32) {
    auto enc = (PFN_cuTensorMapEncodeTiled_v12000)m->ctx->encode_tiled;
    cuuint64_t dims[2] = {(cuuint64_t)rec_floats, (cuuint64_t)m->np};
    cuuint64_t strides[1] = {(cuuint64_t)rec_floats * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)rec_floats, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)rec, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(PB_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return PB_OK;
}

// FP32-pipe operations per point pair by the formula count of the kernels
// above (FADD, FMUL and FFMA each one; the two MUFU operations not counted):
// shared geometry 17, a phi-row 4, a DT-row 15, split coordinates +6.
constexpr double OPS_VK2 = 25.0, OPS_VKDT = 36.0, OPS_SPLIT = 6.0;



// Algorithmic bytes of one gather + near-field SpMV launch: the pattern
// (row pointers, columns) and the four combined block values of every entry
// (value bytes vb each), x and y (2 nv doubles each) once, and with a far
// field the vertex->triangle list and the per-triangle sums (6 doubles).
static double spmv_bytes(const pb_mesh* m, bool far, int vb) {
    const double nv = (double)m->nv, nt = (double)m->nt, nnz = (double)m->nnz;
    double b = 4.0 * (nv + 1.0) + nnz * (4.0 + 4.0 * vb) + 2.0 * 16.0 * nv;
    if (far) b += 4.0 * (nv + 1.0) + 4.0 * 3.0 * nt + 48.0 * nt;
    return b;
}

int apply_blockop(const pb_mesh* m, const pb_near* nf, const BlockOp& B, int prec, const double* x, double* y,
                  cudaStream_t s, const double* comb) {
    if (prec != PB_F64 && prec != PB_F32 && prec != PB_F32_ACCURATE)
        return set_error(PB_EINVAL, "unknown precision %d", prec);
    FarPlan fp;
    PB_TRY(make_far_plan(B, nf->kappa, &fp));
    const int64_t nv = m->nv, nt = m->nt, np = m->np;
    PB_TRY(ws_reserve(const_cast<pb_mesh*>(m)->ws_src, sizeof(float) * REC2 * np + 256));  // >= REC64 doubles
    PB_TRY(ws_reserve(const_cast<pb_mesh*>(m)->ws_tri, sizeof(double) * 6 * nt));
    double* tri = (double*)m->ws_tri.ptr;
    int* status = m->status;
    const double* c64 = comb;
    if (!comb) {
        PB_TRY(ws_reserve(const_cast<pb_mesh*>(m)->ws_comb, (sizeof(double) + sizeof(float)) * 4 * m->nnz));
        double* w64 = (double*)m->ws_comb.ptr;
        PB_TRY(combine_near(m, nf, B, w64, (float*)(w64 + 4 * m->nnz), s));
        c64 = w64;
    }
    const float* c32 = (const float*)(c64 + 4 * m->nnz);

    if (fp.any) {
        bool need_u = false, need_v = false;
        for (int R = 0; R < 2; ++R)
            for (int o = 1; o < O_N; ++o) {
                need_u = need_u || B.c[R][0][o] != 0.0;
                need_v = need_v || B.c[R][1][o] != 0.0;
            }
        const int nacc = fp.mode == 0 ? 2 : 10;
        Rule rule = mesh_rule(m);
        unsigned tb = (unsigned)((nt + 127) / 128);
        if (prec == PB_F64) {
            double* rec = (double*)m->ws_src.ptr;
            k_sources<double, REC64><<<tb, 128, 0, s>>>(nt, m->Q, rule, m->tris, m->tgeo, m->pts64, m->pts32,
                                                        m->pts32lo, x, x + nv, need_u, need_v, rec); ::pb::count_launch();
            const void* kern = fp.mode == 0 ? (const void*)k_pair64<0> : (const void*)k_pair64<1>;
            int S = choose_splits(np, TPB64, TS64, occupancy_slots(m, kern, TPB64));
            int64_t chunk = ((np + S - 1) / S + TS64 - 1) / TS64 * TS64;
            S = (int)((np + chunk - 1) / chunk);
            Coef cf;
            for (int R = 0; R < 2; ++R)
                for (int j = 0; j < 4; ++j) cf.k[R][j] = fp.k[R][j];
            cf.kappa = fp.kappa;
            dim3 grid((unsigned)((np + TPB64 - 1) / TPB64), (unsigned)S);
            PB_TRY(ws_reserve(const_cast<pb_mesh*>(m)->ws_part, sizeof(double) * (size_t)S * nacc * np));
            double* part = (double*)m->ws_part.ptr;
            Timer tm(m->ctx, PB_KERNEL_PAIR64, s, (double)np * (double)np, fp.mode == 0 ? OPS_VK2 : OPS_VKDT);
            if (fp.mode == 0) k_pair64<0><<<grid, TPB64, 0, s>>>(np, m->pts64, rec, cf, chunk, part);
            else k_pair64<1><<<grid, TPB64, 0, s>>>(np, m->pts64, rec, cf, chunk, part);
            ::pb::count_launch();
            tm.stop();
            k_tri_reduce<double><<<tb, 128, 0, s>>>(nt, np, rule, S, fp.mode, fp, m->tgeo, m->pts64, part, tri);
            ::pb::count_launch();
        } else if (prec == PB_F32 && m->ctx->tree_enable && np >= m->ctx->tree_min_points && np > 256) {
            // treecode far field (inner iterations)
            float* part = nullptr;
            int S = 1;
            PB_TRY(tree_far(m, fp, x, need_u, need_v, &part, &S, s));
            k_tri_reduce<float><<<tb, 128, 0, s>>>(nt, np, rule, S, fp.mode, fp, m->tgeo, m->pts64, part, tri);
            ::pb::count_launch();
        } else if (tuned(m->ctx, np, fp.mode, prec == PB_F32_ACCURATE).kernel == 2 ||
                   (tuned(m->ctx, np, fp.mode, prec == PB_F32_ACCURATE).kernel == 0 && m->ctx->pair_kernel == 2)) {
            float* rec = (float*)m->ws_src.ptr;
            k_sources2<float><<<tb, 128, 0, s>>>(nt, m->Q, rule, m->tris, m->tgeo, m->pts64, m->pts32, m->pts32lo, x,
                                                 x + nv, need_u, need_v, rec);
            ::pb::count_launch();
            bool acc = prec == PB_F32_ACCURATE;
            const TuneEntry te = tuned(m->ctx, np, fp.mode, acc);
            const X2Entry& xk = x2_kernel(fp.mode, acc, te.shape);
            CUtensorMap map;
            PB_TRY(make_tmap(m, rec, &map, REC2, xk.ts));
            const int tpc = TPB2 * 2 * xk.npk;
            int S = choose_splits(np, tpc, xk.ts, occupancy_slots(m, xk.fn, TPB2));
            S = scaled_splits(S, te.split_scale, np, xk.ts);
            int64_t chunk = ((np + S - 1) / S + xk.ts - 1) / xk.ts * xk.ts;
            S = (int)((np + chunk - 1) / chunk);
            Coef32 cf;
            for (int R = 0; R < 2; ++R)
                for (int j = 0; j < 4; ++j) cf.k[R][j] = (float)fp.k[R][j];
            cf.kappa = (float)fp.kappa;
            cf.mk2 = (float)(-fp.kappa * 1.4426950408889634);
            dim3 grid((unsigned)((np + tpc - 1) / tpc), (unsigned)S);
            PB_TRY(ws_reserve(const_cast<pb_mesh*>(m)->ws_part, (acc ? sizeof(double) : sizeof(float)) * (size_t)S * nacc * np));
            void* part = m->ws_part.ptr;
            double ops = (fp.mode == 0 ? OPS_VK2 : OPS_VKDT) + (acc ? OPS_SPLIT : 0.0);
            Timer tm(m->ctx, acc ? PB_KERNEL_PAIR32_ACCURATE : PB_KERNEL_PAIR32, s, (double)np * (double)np, ops);
            xk.launch(grid, s, map, np, m->pts32, m->pts32lo, cf, chunk, part, status);
            ::pb::count_launch();
            tm.stop();
            if (acc)
                k_tri_reduce<double><<<tb, 128, 0, s>>>(nt, np, rule, S, fp.mode, fp, m->tgeo, m->pts64,
                                                        (const double*)part, tri);
            else
                k_tri_reduce<float><<<tb, 128, 0, s>>>(nt, np, rule, S, fp.mode, fp, m->tgeo, m->pts64,
                                                       (const float*)part, tri);
            ::pb::count_launch();
        } else {
            float* rec = (float*)m->ws_src.ptr;
            k_sources<float, REC32><<<tb, 128, 0, s>>>(nt, m->Q, rule, m->tris, m->tgeo, m->pts64, m->pts32,
                                                       m->pts32lo, x, x + nv, need_u, need_v, rec);
            ::pb::count_launch();
            CUtensorMap map;
            PB_TRY(make_tmap(m, rec, &map));
            bool acc = prec == PB_F32_ACCURATE;
            const void* kern = fp.mode == 0 ? (acc ? (const void*)k_pair32<0, true> : (const void*)k_pair32<0, false>)
                                            : (acc ? (const void*)k_pair32<1, true> : (const void*)k_pair32<1, false>);
            int S = choose_splits(np, TPB32 * TGT32, TS32, occupancy_slots(m, kern, TPB32));
            S = scaled_splits(S, tuned(m->ctx, np, fp.mode, acc).split_scale, np, TS32);
            int64_t chunk = ((np + S - 1) / S + TS32 - 1) / TS32 * TS32;
            S = (int)((np + chunk - 1) / chunk);
            Coef32 cf;
            for (int R = 0; R < 2; ++R)
                for (int j = 0; j < 4; ++j) cf.k[R][j] = (float)fp.k[R][j];
            cf.kappa = (float)fp.kappa;
            cf.mk2 = (float)(-fp.kappa * 1.4426950408889634);
            dim3 grid((unsigned)((np + TPB32 * TGT32 - 1) / (TPB32 * TGT32)), (unsigned)S);
            PB_TRY(ws_reserve(const_cast<pb_mesh*>(m)->ws_part, (acc ? sizeof(double) : sizeof(float)) * (size_t)S * nacc * np));
            void* part = m->ws_part.ptr;
            double ops = (fp.mode == 0 ? OPS_VK2 : OPS_VKDT) + (acc ? OPS_SPLIT : 0.0);
            Timer tm(m->ctx, acc ? PB_KERNEL_PAIR32_ACCURATE : PB_KERNEL_PAIR32, s, (double)np * (double)np, ops);
            if (fp.mode == 0) {
                if (acc) k_pair32<0, true><<<grid, TPB32, 0, s>>>(map, np, m->pts32, m->pts32lo, cf, chunk, part, status);
                else k_pair32<0, false><<<grid, TPB32, 0, s>>>(map, np, m->pts32, m->pts32lo, cf, chunk, part, status);
            } else {
                if (acc) k_pair32<1, true><<<grid, TPB32, 0, s>>>(map, np, m->pts32, m->pts32lo, cf, chunk, part, status);
                else k_pair32<1, false><<<grid, TPB32, 0, s>>>(map, np, m->pts32, m->pts32lo, cf, chunk, part, status);
            }
            ::pb::count_launch();
            tm.stop();
            if (acc)
                k_tri_reduce<double><<<tb, 128, 0, s>>>(nt, np, rule, S, fp.mode, fp, m->tgeo, m->pts64,
                                                        (const double*)part, tri);
            else
                k_tri_reduce<float><<<tb, 128, 0, s>>>(nt, np, rule, S, fp.mode, fp, m->tgeo, m->pts64,
                                                       (const float*)part, tri);
            ::pb::count_launch();
        }
    }
    unsigned gb = (unsigned)((nv * 8 + 255) / 256);
    Timer tm(m->ctx, PB_KERNEL_SPMV, s, spmv_bytes(m, fp.any, prec == PB_F32 ? 4 : 8), 1.0);
    if (prec == PB_F32)
        k_gather_spmv<float><<<gb, 256, 0, s>>>(nv, m->v2t_ptr, m->v2t, tri, fp.any ? 1 : 0, m->row_ptr, m->col,
                                                c32, m->nnz, x, y);
    else
        k_gather_spmv<double><<<gb, 256, 0, s>>>(nv, m->v2t_ptr, m->v2t, tri, fp.any ? 1 : 0, m->row_ptr, m->col,
                                                 c64, m->nnz, x, y);
    ::pb::count_launch();
    tm.stop();
    PB_CUDA(cudaGetLastError());
    return PB_OK;
}

// y_j = B_j x_j for many meshes: sources per job, one persistent packed
// pair-kernel launch per row mode over all jobs' work items, then each job's
// reduction and gather. prec: PB_F32 or PB_F32_ACCURATE (PB_F64 runs the jobs one by one).
int apply_blockops_batched(const std::vector<FarJob>& jobs, int prec, BatchScratch& bs, cudaStream_t s) {
    if (jobs.empty()) return PB_OK;
    if (prec == PB_F64) {
        for (const FarJob& j : jobs) PB_TRY(apply_blockop(j.m, j.nf, j.B, PB_F64, j.x, j.y, j.s ? j.s : s, j.comb));
        return PB_OK;
    }
    while (bs.ev.size() < jobs.size()) {
        cudaEvent_t e = nullptr;
        PB_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        bs.ev.push_back(e);
    }
    if (!bs.ev_main) PB_CUDA(cudaEventCreateWithFlags(&bs.ev_main, cudaEventDisableTiming));
    if (prec != PB_F32 && prec != PB_F32_ACCURATE) return set_error(PB_EINVAL, "unknown precision %d", prec);
    const bool acc = prec == PB_F32_ACCURATE;
    const int tpc = TPB2 * (acc ? 2 : 4);
    struct Prep {
        FarPlan fp;
        int S;
        int64_t chunk;
        double* tri;
        double* c64;
        float* c32;
    };
    std::vector<Prep> prep(jobs.size());
    std::vector<PairJob> hjobs[2];
    std::vector<int> hjob_of[2];
    std::vector<TreeJob> tjobs[2];
    std::vector<int> tjob_of[2];
    for (size_t k = 0; k < jobs.size(); ++k) {
        const FarJob& J = jobs[k];
        pb_mesh* m = const_cast<pb_mesh*>(J.m);
        Prep& P = prep[k];
        cudaStream_t js = J.s ? J.s : s;
        PB_TRY(make_far_plan(J.B, J.nf->kappa, &P.fp));
        const int64_t nt = m->nt, np = m->np;
        const int64_t np_pad = (np + TS2 - 1) / TS2 * TS2;
        PB_TRY(ws_reserve(m->ws_src, sizeof(float) * REC2 * np_pad + 256));
        PB_TRY(ws_reserve(m->ws_tri, sizeof(double) * 6 * nt));
        P.tri = (double*)m->ws_tri.ptr;
        if (J.comb) {
            P.c64 = const_cast<double*>(J.comb);
        } else {
            PB_TRY(ws_reserve(m->ws_comb, (sizeof(double) + sizeof(float)) * 4 * m->nnz));
            P.c64 = (double*)m->ws_comb.ptr;
            PB_TRY(combine_near(m, J.nf, J.B, P.c64, (float*)(P.c64 + 4 * m->nnz), js));
        }
        P.c32 = (float*)(P.c64 + 4 * m->nnz);
        if (!P.fp.any) continue;
        bool need_u = false, need_v = false;
        for (int R = 0; R < 2; ++R)
            for (int o = 1; o < O_N; ++o) {
                need_u = need_u || J.B.c[R][0][o] != 0.0;
                need_v = need_v || J.B.c[R][1][o] != 0.0;
            }
        if (!acc && m->ctx->tree_enable && np >= m->ctx->tree_min_points && np > 256) {
            // treecode: its sources and proxy charges now, its leaves in the shared launch
            TreeJob tj;
            PB_TRY(tree_prepare(m, P.fp, J.x, need_u, need_v, &tj, js));
            P.S = tj.nsplit;
            tjobs[P.fp.mode].push_back(tj);
            tjob_of[P.fp.mode].push_back((int)k);
            continue;
        }
        float* rec = (float*)m->ws_src.ptr;
        unsigned tb = (unsigned)((nt + 127) / 128);
        k_sources2<float><<<tb, 128, 0, js>>>(nt, m->Q, mesh_rule(m), m->tris, m->tgeo, m->pts64, m->pts32,
                                              m->pts32lo, J.x, J.x + m->nv, need_u, need_v, rec);
        ::pb::count_launch();
        if (np_pad > np) PB_CUDA(cudaMemsetAsync(rec + REC2 * np, 0, sizeof(float) * REC2 * (np_pad - np), js));
        // the single-mesh decomposition (same kernel occupancy as that path)
        const void* kern = x2_kernel(P.fp.mode, acc, 0).fn;  // the default shape's occupancy (the batched kernel's)
        int S = choose_splits(np, tpc, TS2, occupancy_slots(m, kern, TPB2));
        S = scaled_splits(S, tuned(m->ctx, np, P.fp.mode, acc).split_scale, np, TS2);
        P.chunk = ((np + S - 1) / S + TS2 - 1) / TS2 * TS2;
        P.S = (int)((np + P.chunk - 1) / P.chunk);
        const int nacc = P.fp.mode == 0 ? 2 : 10;
        PB_TRY(ws_reserve(m->ws_part, (acc ? sizeof(double) : sizeof(float)) * (size_t)P.S * nacc * np));
        PairJob pj;
        pj.rec = rec;
        pj.pts32 = m->pts32;
        pj.pts32lo = m->pts32lo;
        pj.part = m->ws_part.ptr;
        pj.np = np;
        pj.chunk = P.chunk;
        for (int R = 0; R < 2; ++R)
            for (int j = 0; j < 4; ++j) pj.cf.k[R][j] = (float)P.fp.k[R][j];
        pj.cf.kappa = (float)P.fp.kappa;
        pj.cf.mk2 = (float)(-P.fp.kappa * 1.4426950408889634);
        pj.nsplit = P.S;
        pj.pad = 0;
        hjobs[P.fp.mode].push_back(pj);
        hjob_of[P.fp.mode].push_back((int)k);
    }
    // the jobs' own streams' work (sources, near values, tree preparation) before the shared launch
    for (size_t k = 0; k < jobs.size(); ++k)
        if (jobs[k].s && jobs[k].s != s) {
            PB_CUDA(cudaEventRecord(bs.ev[k], jobs[k].s));
            PB_CUDA(cudaStreamWaitEvent(s, bs.ev[k], 0));
        }
    for (int mode = 0; mode < 2; ++mode) {
        if (hjobs[mode].empty() && tjobs[mode].empty()) continue;
        // work items, the most expensive first (longest processing time first): a pair item
        // costs its target block times its split's sources; a tree item the average pairs of
        // its tree's leaves and splits, weighted by the tree kernel's lower rate per pair
        std::vector<std::pair<double, PairItem>> costed;
        for (size_t q = 0; q < hjobs[mode].size(); ++q) {
            const PairJob& pj = hjobs[mode][q];
            const int ntb = (int)((pj.np + tpc - 1) / tpc);
            for (int sp = 0; sp < pj.nsplit; ++sp) {
                const int64_t j0 = sp * pj.chunk, j1 = std::min(pj.np, j0 + pj.chunk);
                const double cost = (double)tpc * (double)((j1 - j0 + TS2 - 1) / TS2 * TS2);
                for (int tb = 0; tb < ntb; ++tb) costed.push_back({cost, {(int)q, tb, sp, 0}});
            }
        }
        for (size_t q = 0; q < tjobs[mode].size(); ++q) {
            const pb_mesh* tm_ = jobs[tjob_of[mode][q]].m;
            const TreeJob& tj = tjobs[mode][q];
            const int64_t nleaf = tree_leaves(tm_);
            const double cost = 1.4 * (double)tree_interactions(tm_) / (double)std::max<int64_t>(1, nleaf * tj.nsplit);
            for (int64_t leaf = 0; leaf < nleaf; ++leaf)
                for (int sp = 0; sp < tj.nsplit; ++sp) costed.push_back({cost, {(int)q, (int)leaf, sp, 1}});
        }
        std::stable_sort(costed.begin(), costed.end(),
                         [](const std::pair<double, PairItem>& a, const std::pair<double, PairItem>& b) {
                             return a.first > b.first;
                         });
        std::vector<PairItem> items(costed.size());
        for (size_t i = 0; i < costed.size(); ++i) items[i] = costed[i].second;
        const size_t jb = sizeof(PairJob) * hjobs[mode].size(), tjb = sizeof(TreeJob) * tjobs[mode].size();
        const size_t ib = sizeof(PairItem) * items.size();
        const size_t jb_al = (jb + 255) / 256 * 256, tjb_al = (tjb + 255) / 256 * 256, ib_al = (ib + 255) / 256 * 256;
        PB_TRY(ws_reserve(bs.table, jb_al + tjb_al + ib_al + 256));
        char* base = (char*)bs.table.ptr;
        PairJob* djobs = (PairJob*)base;
        TreeJob* dtjobs = (TreeJob*)(base + jb_al);
        PairItem* ditems = (PairItem*)(base + jb_al + tjb_al);
        int* counter = (int*)(base + jb_al + tjb_al + ib_al);
        if (jb) PB_CUDA(cudaMemcpyAsync(djobs, hjobs[mode].data(), jb, cudaMemcpyHostToDevice, s));
        if (tjb) PB_CUDA(cudaMemcpyAsync(dtjobs, tjobs[mode].data(), tjb, cudaMemcpyHostToDevice, s));
        PB_CUDA(cudaMemcpyAsync(ditems, items.data(), ib, cudaMemcpyHostToDevice, s));
        PB_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), s));
        int* status = jobs[hjob_of[mode].empty() ? tjob_of[mode][0] : hjob_of[mode][0]].m->status;
        const int n_items = (int)items.size();
        const void* kern = mode == 0 ? (acc ? (const void*)k_pair32x2_queue<0, true> : (const void*)k_pair32x2_queue<0, false>)
                                     : (acc ? (const void*)k_pair32x2_queue<1, true> : (const void*)k_pair32x2_queue<1, false>);
        const pb_ctx* ctx = jobs[hjob_of[mode].empty() ? tjob_of[mode][0] : hjob_of[mode][0]].m->ctx;
        int per_sm = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TPB2, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
        cudaGetLastError();
        const unsigned grid = (unsigned)std::max(1, std::min(n_items, per_sm * ctx->num_sms));
        if (mode == 0) {
            if (acc) k_pair32x2_queue<0, true><<<grid, TPB2, 0, s>>>(djobs, dtjobs, ditems, n_items, counter, status);
            else k_pair32x2_queue<0, false><<<grid, TPB2, 0, s>>>(djobs, dtjobs, ditems, n_items, counter, status);
        } else {
            if (acc) k_pair32x2_queue<1, true><<<grid, TPB2, 0, s>>>(djobs, dtjobs, ditems, n_items, counter, status);
            else k_pair32x2_queue<1, false><<<grid, TPB2, 0, s>>>(djobs, dtjobs, ditems, n_items, counter, status);
        }
        ::pb::count_launch();
    }
    // and the shared launch before the jobs' own reductions
    PB_CUDA(cudaEventRecord(bs.ev_main, s));
    for (size_t k = 0; k < jobs.size(); ++k)
        if (jobs[k].s && jobs[k].s != s) PB_CUDA(cudaStreamWaitEvent(jobs[k].s, bs.ev_main, 0));
    for (size_t k = 0; k < jobs.size(); ++k) {
        const FarJob& J = jobs[k];
        const pb_mesh* m = J.m;
        const Prep& P = prep[k];
        cudaStream_t js = J.s ? J.s : s;
        if (P.fp.any) {
            unsigned tb = (unsigned)((m->nt + 127) / 128);
            if (acc)
                k_tri_reduce<double><<<tb, 128, 0, js>>>(m->nt, m->np, mesh_rule(m), P.S, P.fp.mode, P.fp, m->tgeo,
                                                         m->pts64, (const double*)m->ws_part.ptr, P.tri);
            else
                k_tri_reduce<float><<<tb, 128, 0, js>>>(m->nt, m->np, mesh_rule(m), P.S, P.fp.mode, P.fp, m->tgeo,
                                                        m->pts64, (const float*)m->ws_part.ptr, P.tri);
            ::pb::count_launch();
        }
        unsigned gb = (unsigned)((m->nv * 8 + 255) / 256);
        if (prec == PB_F32)
            k_gather_spmv<float><<<gb, 256, 0, js>>>(m->nv, m->v2t_ptr, m->v2t, P.tri, P.fp.any ? 1 : 0, m->row_ptr,
                                                     m->col, P.c32, m->nnz, J.x, J.y);
        else
            k_gather_spmv<double><<<gb, 256, 0, js>>>(m->nv, m->v2t_ptr, m->v2t, P.tri, P.fp.any ? 1 : 0,
                                                      m->row_ptr, m->col, P.c64, m->nnz, J.x, J.y);
        ::pb::count_launch();
    }
    PB_CUDA(cudaGetLastError());
    return PB_OK;
}

void batch_scratch_free(BatchScratch& bs) {
    ws_free(bs.table);
    for (cudaEvent_t e : bs.ev) cudaEventDestroy(e);
    bs.ev.clear();
    if (bs.ev_main) cudaEventDestroy(bs.ev_main);
    bs.ev_main = nullptr;
}

int far_splits_estimate(pb_ctx* ctx, int64_t np) {
    int best = 1;
    const void* kerns[2] = {x2_kernel(1, true, 0).fn, x2_kernel(1, false, 0).fn};
    const int tpcs[2] = {TPB2 * 2, TPB2 * 4};
    for (int k = 0; k < 2; ++k) {
        int per_sm = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kerns[k], TPB2, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        cudaGetLastError();
        best = std::max(best, choose_splits(np, tpcs[k], TS2, per_sm * ctx->num_sms));
    }
    return best;
}

int far_splits(const pb_mesh* m, int tpc, int ctas_per_sm) {
    return choose_splits(m->np, tpc, TS32, ctas_per_sm * m->ctx->num_sms);
}

}  // namespace pb

// ------------------------------------------------------ allocation-free variant
// Some callers cannot call cudaMalloc: a process whose device memory is owned
// entirely by another allocator (a framework that reserves almost all of HBM
// up front, so a raw cudaMalloc fails or steals from it), or a latency-bound
// loop that must not pay for the device-wide synchronisation that cudaMalloc
// and cudaFree imply. pb_system_apply_noalloc serves them: the FP32 system
// application with every temporary in the file-scope array below instead of
// the mesh's workspaces.
namespace pb {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;  // 16 MiB on every GPU that loads the library
constexpr int NOALLOC_MAX_SPLITS = 4;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array, looked up once per device. In host code
// the array's name is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress with that device current.
static int noalloc_scratch(int device, unsigned char** out) {
    static std::mutex mu;
    static unsigned char* addr[64] = {nullptr};
    if (device < 0 || device >= 64) return set_error(PB_EINVAL, "device %d out of range", device);
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(PB_ECUDA, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
        addr[device] = (unsigned char*)p;
    }
    *out = addr[device];
    return PB_OK;
}

static size_t align256(size_t n) { return (n + 255) / 256 * 256; }

}  // namespace pb

extern "C" int pb_system_apply_noalloc(pb_ctx* ctx, const pb_mesh* m, const pb_near* nf, const pb_params* prm,
                                       int form, double alpha, double beta, const double* x, double* y,
                                       void* stream) {
    using namespace pb;
    if (!ctx || !m || !nf || !prm || !x || !y) return set_error(PB_EINVAL, "pb_system_apply_noalloc: NULL argument");
    if (nf->mesh != m) return set_error(PB_EINVAL, "near field belongs to another mesh");
    if (m->ctx != ctx) return set_error(PB_EINVAL, "pb_system_apply_noalloc: the mesh was loaded in another context");
    if (x == y) return set_error(PB_EINVAL, "x and y must not overlap");
    BlockOp B;
    PB_TRY(system_blockop(prm, form, alpha, beta, &B));
    FarPlan fp;
    PB_TRY(make_far_plan(B, nf->kappa, &fp));
    const int64_t nv = m->nv, nt = m->nt, np = m->np;
    const int nacc = fp.mode == 0 ? 2 : 10;
    // scratch layout: sources | partial sums (<= 4 splits) | per-triangle sums | combined near values
    const size_t b_src = align256(sizeof(float) * REC32 * (size_t)np);
    const size_t b_part = align256(sizeof(float) * NOALLOC_MAX_SPLITS * 10 * (size_t)np);
    const size_t b_tri = align256(sizeof(double) * 6 * (size_t)nt);
    const size_t b_comb = align256((sizeof(double) + sizeof(float)) * 4 * (size_t)m->nnz);
    const size_t need = b_src + b_part + b_tri + b_comb;
    if (need > NOALLOC_SCRATCH_BYTES)
        return set_error(PB_EINVAL, "pb_system_apply_noalloc: mesh needs %zu bytes of scratch, the limit is %zu "
                         "(%lld triangles here)", need, NOALLOC_SCRATCH_BYTES, (long long)nt);
    // the mesh's device: its arrays, tensor map and occupancy queries all live there
    PB_CUDA(cudaSetDevice(m->ctx->device));
    unsigned char* base = nullptr;
    PB_TRY(noalloc_scratch(m->ctx->device, &base));
    float* rec = (float*)base;
    float* part = (float*)(base + b_src);
    double* tri = (double*)(base + b_src + b_part);
    double* c64 = (double*)(base + b_src + b_part + b_tri);
    float* c32 = (float*)(c64 + 4 * m->nnz);
    cudaStream_t s = (cudaStream_t)stream;
    // every scratch word read below is first written by this call: nothing to clear
    PB_TRY(combine_near(m, nf, B, c64, c32, s));
    if (fp.any) {
        bool need_u = false, need_v = false;
        for (int R = 0; R < 2; ++R)
            for (int o = 1; o < O_N; ++o) {
                need_u = need_u || B.c[R][0][o] != 0.0;
                need_v = need_v || B.c[R][1][o] != 0.0;
            }
        Rule rule = mesh_rule(m);
        unsigned tb = (unsigned)((nt + 127) / 128);
        k_sources<float, REC32><<<tb, 128, 0, s>>>(nt, m->Q, rule, m->tris, m->tgeo, m->pts64, m->pts32, m->pts32lo,
                                                   x, x + nv, need_u, need_v, rec);
        ::pb::count_launch();
        CUtensorMap map;
        PB_TRY(make_tmap(m, rec, &map));
        const void* kern = fp.mode == 0 ? (const void*)k_pair32<0, false> : (const void*)k_pair32<1, false>;
        int S = std::min(NOALLOC_MAX_SPLITS, choose_splits(np, TPB32 * TGT32, TS32, occupancy_slots(m, kern, TPB32)));
        int64_t chunk = ((np + S - 1) / S + TS32 - 1) / TS32 * TS32;
        S = (int)((np + chunk - 1) / chunk);
        Coef32 cf;
        for (int R = 0; R < 2; ++R)
            for (int j = 0; j < 4; ++j) cf.k[R][j] = (float)fp.k[R][j];
        cf.kappa = (float)fp.kappa;
        cf.mk2 = (float)(-fp.kappa * 1.4426950408889634);
        dim3 grid((unsigned)((np + TPB32 * TGT32 - 1) / (TPB32 * TGT32)), (unsigned)S);
        if (fp.mode == 0)
            k_pair32<0, false><<<grid, TPB32, 0, s>>>(map, np, m->pts32, m->pts32lo, cf, chunk, part, m->status);
        else
            k_pair32<1, false><<<grid, TPB32, 0, s>>>(map, np, m->pts32, m->pts32lo, cf, chunk, part, m->status);
        ::pb::count_launch();
        k_tri_reduce<float><<<tb, 128, 0, s>>>(nt, np, rule, S, fp.mode, fp, m->tgeo, m->pts64, part, tri);
        ::pb::count_launch();
    }
    (void)nacc;
    unsigned gb = (unsigned)((nv * 8 + 255) / 256);
    k_gather_spmv<float><<<gb, 256, 0, s>>>(nv, m->v2t_ptr, m->v2t, tri, fp.any ? 1 : 0, m->row_ptr, m->col, c32,
                                            m->nnz, x, y);
    ::pb::count_launch();
    PB_CUDA(cudaGetLastError());
    return PB_OK;
}

// ------------------------------------------------------------------ a12: autotuner
// Times the FP32 far-field application of one formulation on the caller's
// mesh for every candidate launch (the scalar kernel, or the packed kernel in
// each of its launch shapes - records per TMA tile, pipeline stages, targets
// per thread; split count x0.5, x1, x2 of the wave-filling choice; both the
// fast and the split-coordinate variant), keeps the fastest per variant in the
// context's table for this size bucket, and reports the gain. Results of the
// tuned launches are the same sums in another split and tile order (FP32
// rounding differences only).
extern "C" int pb_autotune(pb_ctx* ctx, const pb_mesh* m, const pb_near* nf, const pb_params* prm, int form,
                           pb_tune_result* out, void* stream) {
    using namespace pb;
    if (!ctx || !m || !nf || !prm) return set_error(PB_EINVAL, "pb_autotune: NULL argument");
    BlockOp B;
    PB_TRY(system_blockop(prm, form, 0.0, 0.0, &B));
    FarPlan fp;
    PB_TRY(make_far_plan(B, nf->kappa, &fp));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n2 = 2 * m->nv;
    double* xy = nullptr;
    PB_TRY(dev_alloc((void**)&xy, sizeof(double) * 2 * n2));
    std::vector<double> hx(n2);
    for (int64_t i = 0; i < n2; ++i) hx[i] = std::sin(0.37 * (double)i) + 0.5;
    cudaMemcpy(xy, hx.data(), sizeof(double) * n2, cudaMemcpyHostToDevice);
    const int bucket = tune_bucket(m->np);
    // candidates: (kernel, shape): the packed kernel in every shape, then the scalar kernel
    std::vector<std::pair<int, int>> cands;
    for (int sh = 0; sh < X2_SHAPES; ++sh) cands.push_back({2, sh});
    cands.push_back({1, 0});
    const double scales[3] = {1.0, 0.5, 2.0};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = PB_OK;
    // the pair kernel is what is timed: the treecode, which would otherwise take the fast
    // variant's applications of large meshes, is off meanwhile
    const int tree_was = ctx->tree_enable;
    ctx->tree_enable = 0;
    for (int acc = 0; acc < 2 && rc == PB_OK; ++acc) {
        const int prec = acc ? PB_F32_ACCURATE : PB_F32;
        TuneEntry& slot = ctx->tune[fp.mode ? 1 : 0][acc][bucket];
        const TuneEntry saved = slot;
        double best = 1e300, dflt = 0.0;
        TuneEntry best_e;
        for (size_t ci = 0; ci < cands.size() && rc == PB_OK; ++ci)
            for (double sc : scales) {
                const auto& kc = cands[ci];
                const int k = kc.first;
                slot.kernel = k;
                slot.shape = kc.second;
                slot.split_scale = sc;
                const uint64_t gen0 = m->ws_gen;
                cudaEventRecord(e0, s);
                rc = apply_blockop(m, nf, B, prec, xy, xy + n2, s);  // warm-up and workspace growth
                if (rc != PB_OK) break;
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms_total = 0.0f;
                cudaEventElapsedTime(&ms_total, e0, e1);
                // long launches: one timed run each, or none when the warm-up grew no workspace
                // (its time is then a clean measurement)
                const int reps = ms_total > 50.0f ? (m->ws_gen == gen0 ? 0 : 1) : 3;
                if (reps > 0) {
                    cudaEventRecord(e0, s);
                    for (int r = 0; r < reps && rc == PB_OK; ++r) rc = apply_blockop(m, nf, B, prec, xy, xy + n2, s);
                    cudaEventRecord(e1, s);
                    cudaEventSynchronize(e1);
                    cudaEventElapsedTime(&ms_total, e0, e1);
                }
                const double ms = ms_total / std::max(1, reps);
                if (k == 2 && kc.second == 0 && sc == 1.0) dflt = ms;
                if (ms < best) {
                    best = ms;
                    best_e = slot;
                }
            }
        slot = rc == PB_OK ? best_e : saved;
        if (out) {
            pb_tune_choice& o = acc ? out->accurate : out->fast;
            o.kernel = best_e.kernel;
            o.shape = best_e.shape;
            const X2Entry& xk = x2_kernel(fp.mode, acc != 0, best_e.shape);
            o.tile_records = best_e.kernel == 2 ? xk.ts : (int)TS32;
            o.stages = best_e.kernel == 2 ? xk.st : (int)ST32;
            o.targets_per_thread = best_e.kernel == 2 ? 2 * xk.npk : (int)TGT32;
            o.tiles_per_fp64_sum = best_e.kernel == 2 && acc ? xk.promo : 1;
            o.split_scale = best_e.split_scale;
            o.best_ms = best;
            o.default_ms = dflt;
        }
    }
    ctx->tree_enable = tree_was;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(xy);
    if (rc == PB_OK) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = set_error(PB_ECUDA, "pb_autotune: %s", cudaGetErrorString(e));
    }
    return rc;
}

// -------------------------------------------------- failure detection self-test
// The bounded mbarrier wait of the pair kernels, on a barrier that nothing
// arrives at and no copy targets: after `polls` polls the wait gives up,
// records PB_ETIMEOUT in the status word and the kernel returns normally.
namespace pb {
__global__ void k_wait_selftest(int64_t polls, int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    bool done = false;
    for (int64_t i = 0; i < polls && !done; ++i) done = mbar_try_wait(&bar, 0);
    if (!done && threadIdx.x == 0) atomicExch(status, PB_ETIMEOUT);
}
}  // namespace pb

extern "C" int pb_selftest_wait(pb_ctx* ctx, int64_t polls, int* status_out) {
    using namespace pb;
    if (!ctx || !status_out || polls < 1 || polls > ((int64_t)1 << 24))
        return set_error(PB_EINVAL, "pb_selftest_wait: bad argument");
    PB_CUDA(cudaSetDevice(ctx->device));
    int* st = nullptr;
    PB_TRY(dev_alloc((void**)&st, sizeof(int)));
    cudaMemset(st, 0, sizeof(int));
    k_wait_selftest<<<1, 32>>>(polls, st);
    ::pb::count_launch();
    cudaError_t e = cudaMemcpy(status_out, st, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(st);
    if (e != cudaSuccess) return set_error(PB_ECUDA, "pb_selftest_wait: %s", cudaGetErrorString(e));
    return PB_OK;
}

// ----------------------------------------------- arithmetic peak microbenchmark
// Independent fused multiply-add chains (eight per thread, so that the pipe,
// not the dependency latency, sets the rate) on a grid of four CTAs per SM:
// the issue rate the roofline of the pair and near-field kernels is measured
// against. The chains' sum is stored only when it equals an impossible value,
// so the compiler keeps every FMA.
namespace pb {
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, T b, T c, T* __restrict__ out) {
    T a[8];
    for (int k = 0; k < 8; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
    }
    T t = 0;
    for (int k = 0; k < 8; ++k) t += a[k];
    if (t == (T)-12345.0) out[0] = t;
}
__global__ void __launch_bounds__(256) k_fma2_peak(int iters, float b, float c, float* __restrict__ out) {
    float2 a[8];
    for (int k = 0; k < 8; ++k) a[k] = make_float2((threadIdx.x + k) * 1e-3f, (threadIdx.x - k) * 1e-3f);
    const float2 bb = splat(b), cc = splat(c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = fma2(a[k], bb, cc);
    }
    float t = 0;
    for (int k = 0; k < 8; ++k) t += a[k].x + a[k].y;
    if (t == -12345.0f) out[0] = t;
}
}  // namespace pb

extern "C" int pb_measure_peak(pb_ctx* ctx, int kind, double* fma_per_s) {
    using namespace pb;
    if (!ctx || !fma_per_s || kind < 0 || kind > 2) return set_error(PB_EINVAL, "pb_measure_peak: bad argument");
    PB_CUDA(cudaSetDevice(ctx->device));
    double* out = nullptr;
    PB_TRY(dev_alloc((void**)&out, 64));
    const unsigned blocks = (unsigned)(4 * ctx->num_sms);
    // about 20 ms per launch at the nominal rates
    const int iters = kind == 1 ? 600 : 40000;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {  // the first launch warms up
        cudaEventRecord(e0);
        if (kind == 0) k_fma_peak<float><<<blocks, 256>>>(iters, 0.999999f, 1e-7f, (float*)out);
        else if (kind == 1) k_fma_peak<double><<<blocks, 256>>>(iters, 0.999999, 1e-7, out);
        else k_fma2_peak<<<blocks, 256>>>(iters / 2, 0.999999f, 1e-7f, (float*)out);
        ::pb::count_launch();
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(PB_ECUDA, "pb_measure_peak: %s", cudaGetErrorString(e));
    // FMAs per launch: threads x iterations x 16 x 8 chains (x 2 lanes for f32x2 at half the iterations)
    const double fmas = (double)blocks * 256.0 * (double)iters * 128.0;
    *fma_per_s = fmas / (best * 1e-3);
    return PB_OK;
}
