// a6 + a10: charges -> surface (right-hand side) and surface -> charges
// (reaction potential, solvation energy), FP64.
//
// Paper eq. sources: phi_D(x) = sum_j q_j / (4 pi eps_int |x - x_j|) and
// phi_N = d phi_D / dn_x, tested against the P1 basis with the far rule.
// Paper eqs. phireac_bie and dG: phi_reac(x_j) = V_int[v_int](x_j) - K_int[u_int](x_j),
// Delta G = 1/2 sum_j q_j phi_reac(x_j).
#include <math.h>

#include <cmath>

#include "internal.h"

namespace pb {

int rhs_coefs(const pb_params* prm, int form, double alpha, double beta, double d[2], double n[2]);

constexpr int QTILE = 256;

// 1/sqrt(x) in FP64 for x in the normal FP32 range (squared distances here):
// the FP32 hardware estimate (relative error below 2^-22) refined by two
// Newton steps for f(y) = y^-2 - x, y <- y + y (1 - x y^2) / 2; each step squares
// the relative error (2^-44, then rounding level), about 2 ulp in all.
__device__ __forceinline__ double rsqrt_nr(double x) {
    float yf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(__double2float_rn(x)));
    double y = (double)yf;
    double e = __fma_rn(-(x * y), y, 1.0);
    y = __fma_rn(0.5 * y, e, y);
    e = __fma_rn(-(x * y), y, 1.0);
    return __fma_rn(0.5 * y, e, y);
}

// per point: phi_D and phi_N of all charges, then per triangle the tested sums
// (templated on the rule's point count, so that the per-point sums stay in registers)
template <int Q>
__global__ void k_rhs_points(int64_t nt, Rule rule, const double* __restrict__ pts64, const double* __restrict__ tgeo,
                             const double* __restrict__ xq, const double* __restrict__ q, int64_t nq, double eps_int,
                             double* __restrict__ tri_out) {
    __shared__ double sq[QTILE * 4];
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool live = t < nt;
    double pd[6] = {0, 0, 0, 0, 0, 0}, pn[6] = {0, 0, 0, 0, 0, 0};
    double nx = 0, ny = 0, nz = 0;
    if (live) { nx = tgeo[16 * t]; ny = tgeo[16 * t + 1]; nz = tgeo[16 * t + 2]; }
    for (int64_t j0 = 0; j0 < nq; j0 += QTILE) {
        int cnt = (int)min((int64_t)QTILE, nq - j0);
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            sq[4 * k] = xq[3 * (j0 + k)];
            sq[4 * k + 1] = xq[3 * (j0 + k) + 1];
            sq[4 * k + 2] = xq[3 * (j0 + k) + 2];
            sq[4 * k + 3] = q[j0 + k];
        }
        __syncthreads();
        if (live)
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const double* x = pts64 + 4 * (t * Q + k);
                for (int j = 0; j < cnt; ++j) {
                    double d0 = x[0] - sq[4 * j], d1 = x[1] - sq[4 * j + 1], d2 = x[2] - sq[4 * j + 2];
                    double r2 = d0 * d0 + d1 * d1 + d2 * d2;
                    double rinv = rsqrt_nr(r2);
                    double c = sq[4 * j + 3] * rinv;
                    pd[k] += c;
                    pn[k] -= c * rinv * rinv * (d0 * nx + d1 * ny + d2 * nz);
                }
            }
        __syncthreads();
    }
    if (!live) return;
    const double f = 1.0 / (4.0 * M_PI * eps_int);
    double out[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        double w = pts64[4 * (t * Q + k) + 3] * f;
        for (int a = 0; a < 3; ++a) {
            out[a] += w * rule.l[k][a] * pd[k];
            out[3 + a] += w * rule.l[k][a] * pn[k];
        }
    }
    for (int k = 0; k < 6; ++k) tri_out[6 * t + k] = out[k];
}

// FP32 pair arithmetic on split coordinates (PB_F32_ACCURATE): every position
// is taken relative to the mesh centre c and split into hi = fl32(x - c) and
// lo = fl32(x - c - hi), so that x - y = (hi_x - hi_y) + (lo_x - lo_y) keeps
// about FP32 precision relative to |x - y| even for close pairs; 1/r by the
// FP32 estimate and one Newton step (about 1 ulp).
__device__ __forceinline__ float rsqrt_f32(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    const float e = fmaf(-(x * y), y, 1.0f);
    return fmaf(0.5f * y, e, y);
}
__device__ __forceinline__ void split3(const double* x, const double* c, float* hi, float* lo) {
    for (int k = 0; k < 3; ++k) {
        const double r = x[k] - c[k];
        hi[k] = (float)r;
        lo[k] = (float)(r - (double)hi[k]);
    }
}
struct Ctr {
    double c[3];
};

// the right-hand side's point sums (k_rhs_points) in FP32 on split coordinates:
// per charge tile the sums in FP32, added into FP64 sums per tile
template <int Q>
__global__ void k_rhs_points32(int64_t nt, Rule rule, const double* __restrict__ pts64,
                               const double* __restrict__ tgeo, const double* __restrict__ xq,
                               const double* __restrict__ q, int64_t nq, double eps_int, Ctr ctr,
                               double* __restrict__ tri_out) {
    __shared__ float4 sh[QTILE], sl[QTILE];
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool live = t < nt;
    float xh[Q][3], xl[Q][3];
    float nx = 0.f, ny = 0.f, nz = 0.f;
    if (live) {
        nx = (float)tgeo[16 * t];
        ny = (float)tgeo[16 * t + 1];
        nz = (float)tgeo[16 * t + 2];
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        if (live) split3(pts64 + 4 * (t * Q + k), ctr.c, xh[k], xl[k]);
        else xh[k][0] = xh[k][1] = xh[k][2] = xl[k][0] = xl[k][1] = xl[k][2] = 0.f;
    }
    double pd[Q], pn[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) pd[k] = pn[k] = 0.0;
    for (int64_t j0 = 0; j0 < nq; j0 += QTILE) {
        const int cnt = (int)min((int64_t)QTILE, nq - j0);
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            float h[3], l[3];
            split3(xq + 3 * (j0 + k), ctr.c, h, l);
            sh[k] = make_float4(h[0], h[1], h[2], (float)q[j0 + k]);
            sl[k] = make_float4(l[0], l[1], l[2], 0.f);
        }
        __syncthreads();
        if (live) {
            float fd[Q], fn[Q];
#pragma unroll
            for (int k = 0; k < Q; ++k) fd[k] = fn[k] = 0.f;
            for (int j = 0; j < cnt; ++j) {
                const float4 a = sh[j], b = sl[j];
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    const float d0 = (xh[k][0] - a.x) + (xl[k][0] - b.x);
                    const float d1 = (xh[k][1] - a.y) + (xl[k][1] - b.y);
                    const float d2 = (xh[k][2] - a.z) + (xl[k][2] - b.z);
                    const float r2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
                    const float rinv = rsqrt_f32(r2);
                    const float c = a.w * rinv;
                    fd[k] += c;
                    fn[k] = fmaf(-c * rinv * rinv, fmaf(d0, nx, fmaf(d1, ny, d2 * nz)), fn[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                pd[k] += (double)fd[k];
                pn[k] += (double)fn[k];
            }
        }
        __syncthreads();
    }
    if (!live) return;
    const double f = 1.0 / (4.0 * M_PI * eps_int);
    double out[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        double w = pts64[4 * (t * Q + k) + 3] * f;
        for (int a = 0; a < 3; ++a) {
            out[a] += w * rule.l[k][a] * pd[k];
            out[3 + a] += w * rule.l[k][a] * pn[k];
        }
    }
    for (int k = 0; k < 6; ++k) tri_out[6 * t + k] = out[k];
}

__global__ void k_rhs_gather(int64_t nv, const int32_t* __restrict__ v2t_ptr, const int32_t* __restrict__ v2t,
                             const double* __restrict__ tri, double d0, double d1, double n0, double n1,
                             double* __restrict__ rhs) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nv) return;
    double bd = 0.0, bn = 0.0;
    for (int32_t k = v2t_ptr[i]; k < v2t_ptr[i + 1]; ++k) {
        int32_t ta = v2t[k];
        int64_t t = ta / 3;
        int a = ta - 3 * (int)t;
        bd += tri[6 * t + a];
        bn += tri[6 * t + 3 + a];
    }
    rhs[i] = d0 * bd + n0 * bn;
    rhs[nv + i] = d1 * bd + n1 * bn;
}

// phi_reac: the interior traces at every point of the reference rule once
// (position, w v_int and w u_int n_y), then per charge and chunk of points the
// partial sums of G_L v - dG_L/dn_y u (1/(4 pi) applied at the end).
constexpr int EN_THREADS = 256;
constexpr int EN_CHUNK = 8192;

__global__ void k_energy_points(int64_t nt, Rule rule, const int32_t* __restrict__ tris,
                                const double* __restrict__ tgeo, const double* __restrict__ pts64,
                                const double* __restrict__ x, int64_t nv, double vscale, double* __restrict__ pv) {
    const int Q = rule.Q;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nt * Q) return;
    const int64_t t = i / Q;
    const int k = (int)(i - t * Q);
    const int32_t* f = tris + 3 * t;
    const double u = rule.l[k][0] * x[f[0]] + rule.l[k][1] * x[f[1]] + rule.l[k][2] * x[f[2]];
    const double v = vscale * (rule.l[k][0] * x[nv + f[0]] + rule.l[k][1] * x[nv + f[1]] + rule.l[k][2] * x[nv + f[2]]);
    const double* y = pts64 + 4 * i;
    const double* g = tgeo + 16 * t;
    double* o = pv + 8 * i;
    o[0] = y[0];
    o[1] = y[1];
    o[2] = y[2];
    o[3] = y[3] * v;
    o[4] = y[3] * u * g[0];
    o[5] = y[3] * u * g[1];
    o[6] = y[3] * u * g[2];
    o[7] = 0.0;
}

__global__ void k_energy_part(int64_t np, const double* __restrict__ pv, const double* __restrict__ xq,
                              double* __restrict__ part, int nchunk) {
    __shared__ double red[EN_THREADS / 32];
    const int c = blockIdx.x;
    const int64_t j = blockIdx.y;
    const double qx = xq[3 * j], qy = xq[3 * j + 1], qz = xq[3 * j + 2];
    const int64_t i0 = (int64_t)c * EN_CHUNK, i1 = min(np, i0 + EN_CHUNK);
    double s = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += EN_THREADS) {
        const double4 a = *reinterpret_cast<const double4*>(pv + 8 * i);
        const double4 b = *reinterpret_cast<const double4*>(pv + 8 * i + 4);
        const double d0 = qx - a.x, d1 = qy - a.y, d2 = qz - a.z;
        const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
        const double rinv = rsqrt_nr(r2);
        const double dn = d0 * b.x + d1 * b.y + d2 * b.z;  // w u (x_j - y).n_y
        s += rinv * a.w - rinv * rinv * rinv * dn;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tsum = 0.0;
        for (int w = 0; w < EN_THREADS / 32; ++w) tsum += red[w];
        part[j * nchunk + c] = tsum;
    }
}

// the energy's pair sums in FP32 on split coordinates: the point values once
// as (hi, w v), (lo, 0), (w u n, 0) floats, then a thread per charge over a
// chunk of points staged in shared memory, FP32 sums per tile added in FP64
constexpr int EN32_THREADS = 128;  // charges per block
constexpr int EN32_TILE = 256;     // points per staged tile
constexpr int EN32_CHUNK = 4096;   // points per block

__global__ void k_energy_points32(int64_t nt, Rule rule, const int32_t* __restrict__ tris,
                                  const double* __restrict__ tgeo, const double* __restrict__ pts64,
                                  const double* __restrict__ x, int64_t nv, double vscale, Ctr ctr,
                                  float4* __restrict__ pv) {
    const int Q = rule.Q;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nt * Q) return;
    const int64_t t = i / Q;
    const int k = (int)(i - t * Q);
    const int32_t* f = tris + 3 * t;
    const double u = rule.l[k][0] * x[f[0]] + rule.l[k][1] * x[f[1]] + rule.l[k][2] * x[f[2]];
    const double v = vscale * (rule.l[k][0] * x[nv + f[0]] + rule.l[k][1] * x[nv + f[1]] + rule.l[k][2] * x[nv + f[2]]);
    const double* y = pts64 + 4 * i;
    const double* g = tgeo + 16 * t;
    float h[3], l[3];
    split3(y, ctr.c, h, l);
    pv[3 * i] = make_float4(h[0], h[1], h[2], (float)(y[3] * v));
    pv[3 * i + 1] = make_float4(l[0], l[1], l[2], 0.f);
    pv[3 * i + 2] = make_float4((float)(y[3] * u * g[0]), (float)(y[3] * u * g[1]), (float)(y[3] * u * g[2]), 0.f);
}

__global__ void __launch_bounds__(EN32_THREADS) k_energy_part32(int64_t np, const float4* __restrict__ pv,
                                                                const double* __restrict__ xq, int64_t nq, Ctr ctr,
                                                                double* __restrict__ part, int nchunk) {
    __shared__ float4 tile[3 * EN32_TILE];
    const int64_t j = blockIdx.y * (int64_t)EN32_THREADS + threadIdx.x;
    const bool live = j < nq;
    float qh[3] = {0.f, 0.f, 0.f}, ql[3] = {0.f, 0.f, 0.f};
    if (live) split3(xq + 3 * j, ctr.c, qh, ql);
    const int64_t i0 = (int64_t)blockIdx.x * EN32_CHUNK, i1 = min(np, i0 + EN32_CHUNK);
    double s = 0.0;
    for (int64_t b0 = i0; b0 < i1; b0 += EN32_TILE) {
        const int cnt = (int)min((int64_t)EN32_TILE, i1 - b0);
        __syncthreads();
        for (int k = threadIdx.x; k < 3 * cnt; k += EN32_THREADS) tile[k] = pv[3 * b0 + k];
        __syncthreads();
        float f = 0.f;
        for (int p = 0; p < cnt; ++p) {
            const float4 a = tile[3 * p], b = tile[3 * p + 1], c = tile[3 * p + 2];
            const float d0 = (qh[0] - a.x) + (ql[0] - b.x);
            const float d1 = (qh[1] - a.y) + (ql[1] - b.y);
            const float d2 = (qh[2] - a.z) + (ql[2] - b.z);
            const float r2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
            const float rinv = rsqrt_f32(r2);
            const float dn = fmaf(d0, c.x, fmaf(d1, c.y, d2 * c.z));  // w u (x_j - y).n_y
            f = fmaf(rinv, a.w, fmaf(-rinv * rinv * rinv, dn, f));
        }
        s += (double)f;
    }
    if (live) part[j * nchunk + blockIdx.x] = s;
}

// phi_reac(x_j) per charge (its chunks in order), then Delta G by one thread
// over the charges in order: the summation order is fixed.
__global__ void k_energy_rows(int64_t nq, int nchunk, const double* __restrict__ part, double* __restrict__ phi) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= nq) return;
    double p = 0.0;
    for (int c = 0; c < nchunk; ++c) p += part[j * nchunk + c];
    phi[j] = p * (1.0 / (4.0 * M_PI));
}
__global__ void k_energy_final(int64_t nq, const double* __restrict__ phi_all, const double* __restrict__ q,
                               double* __restrict__ phi, double* __restrict__ dG) {
    double e = 0.0;
    for (int64_t j = 0; j < nq; ++j) {
        const double p = phi_all[j];
        if (phi) phi[j] = p;
        e += q[j] * p;
    }
    dG[0] = 0.5 * e;
}

}  // namespace pb

using namespace pb;

extern "C" int pb_rhs_charges(pb_ctx* ctx, const pb_mesh* m, const double* xq, const double* q, int64_t n_q,
                              const pb_params* prm, int form, double alpha, double beta, double* rhs, int prec,
                              void* stream) {
    if (!ctx || !m || !xq || !q || !rhs || !prm) return set_error(PB_EINVAL, "pb_rhs_charges: NULL argument");
    if (n_q < 1) return set_error(PB_EINVAL, "need at least one charge");
    if (prec != PB_F64 && prec != PB_F32_ACCURATE)
        return set_error(PB_EINVAL, "pb_rhs_charges: precision must be PB_F64 or PB_F32_ACCURATE");
    double d[2], n[2];
    PB_TRY(rhs_coefs(prm, form, alpha, beta, d, n));
    cudaStream_t s = (cudaStream_t)stream;
    PB_TRY(ws_reserve(const_cast<pb_mesh*>(m)->ws_tri, sizeof(double) * 6 * m->nt));
    double* tri = (double*)m->ws_tri.ptr;
    // the plan's reference rule (the band rule when the plan has a band)
    const Rule rr = mesh_ref_rule(m);
    const unsigned nbk = (unsigned)((m->nt + 127) / 128);
    if (prec == PB_F64) {
        if (rr.Q == 6) k_rhs_points<6><<<nbk, 128, 0, s>>>(m->nt, rr, m->pts_ref, m->tgeo, xq, q, n_q, prm->eps_int, tri);
        else if (rr.Q == 3) k_rhs_points<3><<<nbk, 128, 0, s>>>(m->nt, rr, m->pts_ref, m->tgeo, xq, q, n_q, prm->eps_int, tri);
        else k_rhs_points<1><<<nbk, 128, 0, s>>>(m->nt, rr, m->pts_ref, m->tgeo, xq, q, n_q, prm->eps_int, tri);
    } else {
        const Ctr c = {{m->ctr[0], m->ctr[1], m->ctr[2]}};
        if (rr.Q == 6)
            k_rhs_points32<6><<<nbk, 128, 0, s>>>(m->nt, rr, m->pts_ref, m->tgeo, xq, q, n_q, prm->eps_int, c, tri);
        else if (rr.Q == 3)
            k_rhs_points32<3><<<nbk, 128, 0, s>>>(m->nt, rr, m->pts_ref, m->tgeo, xq, q, n_q, prm->eps_int, c, tri);
        else
            k_rhs_points32<1><<<nbk, 128, 0, s>>>(m->nt, rr, m->pts_ref, m->tgeo, xq, q, n_q, prm->eps_int, c, tri);
    }
    ::pb::count_launch();
    k_rhs_gather<<<(unsigned)((m->nv + 255) / 256), 256, 0, s>>>(m->nv, m->v2t_ptr, m->v2t, tri, d[0], d[1], n[0],
                                                                n[1], rhs); ::pb::count_launch();
    PB_CUDA(cudaGetLastError());
    return PB_OK;
}

extern "C" int pb_energy(pb_ctx* ctx, const pb_mesh* m, const double* x, int form, const double* xq, const double* q,
                         int64_t n_q, const pb_params* prm, double* phi, double* dG_paper, double* dG_kcal, int prec,
                         void* stream) {
    if (!ctx || !m || !x || !xq || !q || !prm) return set_error(PB_EINVAL, "pb_energy: NULL argument");
    if (prec != PB_F64 && prec != PB_F32_ACCURATE)
        return set_error(PB_EINVAL, "pb_energy: precision must be PB_F64 or PB_F32_ACCURATE");
    if (n_q < 1) return set_error(PB_EINVAL, "need at least one charge");
    if (form < PB_DIRECT_INT || form > PB_LU) return set_error(PB_EINVAL, "unknown formulation %d", form);
    cudaStream_t s = (cudaStream_t)stream;
    // exterior unknowns -> interior traces: u_int = u_ext, v_int = (eps_ext/eps_int) v_ext
    double vscale = form_is_exterior(form) ? prm->eps_ext / prm->eps_int : 1.0;
    const bool f32 = prec == PB_F32_ACCURATE;
    const int nchunk = (int)((m->np_ref + (f32 ? EN32_CHUNK : EN_CHUNK) - 1) / (f32 ? EN32_CHUNK : EN_CHUNK));
    double* part = nullptr;
    // partial sums, phi per charge, Delta G, then the point values (32-byte aligned)
    const size_t n_part = (size_t)n_q * nchunk, n_head = (n_part + 2 * (size_t)n_q + 1 + 3) / 4 * 4;
    PB_TRY(dev_alloc((void**)&part, sizeof(double) * (n_head + 8 * (size_t)m->np_ref)));
    double* phi_all = part + n_part;
    double* dG = phi_all + n_q;
    double* pv = part + n_head;
    const Rule rr = mesh_ref_rule(m);
    const unsigned pb_ = (unsigned)((m->np_ref + 255) / 256);
    if (f32) {
        const Ctr c = {{m->ctr[0], m->ctr[1], m->ctr[2]}};
        k_energy_points32<<<pb_, 256, 0, s>>>(m->nt, rr, m->tris, m->tgeo, m->pts_ref, x, m->nv, vscale, c,
                                              reinterpret_cast<float4*>(pv));
        const dim3 grid(nchunk, (unsigned)((n_q + EN32_THREADS - 1) / EN32_THREADS));
        k_energy_part32<<<grid, EN32_THREADS, 0, s>>>(m->np_ref, reinterpret_cast<const float4*>(pv), xq, n_q, c, part,
                                                      nchunk);
    } else {
        k_energy_points<<<pb_, 256, 0, s>>>(m->nt, rr, m->tris, m->tgeo, m->pts_ref, x, m->nv, vscale, pv);
        const dim3 grid(nchunk, (unsigned)n_q);
        k_energy_part<<<grid, EN_THREADS, 0, s>>>(m->np_ref, pv, xq, part, nchunk);
    }
    k_energy_rows<<<(unsigned)((n_q + 127) / 128), 128, 0, s>>>(n_q, nchunk, part, phi_all);
    k_energy_final<<<1, 1, 0, s>>>(n_q, phi_all, q, phi, dG);
    ::pb::count_launch(4);
    double h = 0.0;
    cudaError_t e = cudaMemcpyAsync(&h, dG, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(part);
    if (e != cudaSuccess) return set_error(PB_ECUDA, "pb_energy: %s", cudaGetErrorString(e));
    if (dG_paper) *dG_paper = h;
    if (dG_kcal) *dG_kcal = h * 4.0 * M_PI * 332.0636;
    return PB_OK;
}

extern "C" int pb_solvation_energy(pb_ctx* ctx, const double* verts, int64_t n_verts, const int32_t* tris,
                                   int64_t n_tris, const double* xq, const double* q, int64_t n_q,
                                   const pb_params* prm, const pb_quad_plan* plan, int form, int precond,
                                   const pb_solve_opts* opts, double* dG_kcal, pb_solve_info* info, void* stream) {
    if (!ctx || !verts || !tris || !xq || !q || !prm || !dG_kcal)
        return set_error(PB_EINVAL, "pb_solvation_energy: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    pb_mesh* m = nullptr;
    pb_near* nf = nullptr;
    double* buf = nullptr;
    int rc = pb_mesh_load(ctx, verts, n_verts, tris, n_tris, plan, PB_MEM_HOST, &m);
    if (rc == PB_OK) rc = pb_near_build(ctx, m, prm->kappa, &nf, stream);
    if (rc == PB_OK) rc = dev_alloc((void**)&buf, sizeof(double) * (4 * n_q + 4 * m->nv));
    if (rc == PB_OK) {
        double* dxq = buf;
        double* dq = buf + 3 * n_q;
        double* rhs = dq + n_q;
        double* x = rhs + 2 * m->nv;
        cudaError_t e = cudaMemcpyAsync(dxq, xq, sizeof(double) * 3 * n_q, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dq, q, sizeof(double) * n_q, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) rc = set_error(PB_ECUDA, "copy of charges: %s", cudaGetErrorString(e));
        double a = opts ? opts->alpha : 0.0, b = opts ? opts->beta : 0.0;
        const int cprec = opts && opts->precision == PB_MIXED ? PB_F32_ACCURATE : PB_F64;
        if (rc == PB_OK) rc = pb_rhs_charges(ctx, m, dxq, dq, n_q, prm, form, a, b, rhs, cprec, stream);
        if (rc == PB_OK) rc = pb_solve(ctx, m, nf, prm, form, precond, opts, rhs, x, info, stream);
        if (rc == PB_OK) rc = pb_energy(ctx, m, x, form, dxq, dq, n_q, prm, nullptr, nullptr, dG_kcal, cprec, stream);
    }
    if (buf) cudaFree(buf);
    pb_free_near(nf);
    pb_free_mesh(m);
    return rc;
}

// a12, quadrature part: the cheapest plan whose Delta G differs from the
// reference plan's by at most tol_dG relative. Candidates, cheapest first: the
// 3-point far rule with the reference's rule inside a distance band of
// 2, 3, 4 and 6 radii (the far-field work is a quarter of the 6-point rule's;
// the band's near-field work grows with its width); then one Gauss point fewer
// per dimension in the singular rule of one class of pair at a time
// (vertex-adjacent, edge-adjacent, coincident: the classes in order of their
// share of the near-field work on a closed surface), each kept while the plan
// still qualifies. The reference plan itself when nothing qualifies. The
// returned plan names its three singular orders explicitly.
extern "C" int pb_autotune_plan(pb_ctx* ctx, const double* verts, int64_t n_verts, const int32_t* tris,
                                int64_t n_tris, const double* xq, const double* q, int64_t n_q, const pb_params* prm,
                                const pb_quad_plan* reference, int form, int precond, const pb_solve_opts* opts,
                                double tol_dG, pb_quad_plan* out_plan, double* out_change, void* stream) {
    if (!ctx || !verts || !tris || !xq || !q || !prm || !out_plan || !(tol_dG >= 0.0))
        return set_error(PB_EINVAL, "pb_autotune_plan: bad argument");
    pb_quad_plan ref = reference ? *reference : pb_quad_plan{6, 4, 0.0, 6, 0, 0, 0};
    int* cls[3] = {&ref.n_ss_coin, &ref.n_ss_edge, &ref.n_ss_vert};
    for (int c = 0; c < 3; ++c)
        if (*cls[c] == 0) *cls[c] = ref.n_ss;
    double dref = 0.0;
    PB_TRY(pb_solvation_energy(ctx, verts, n_verts, tris, n_tris, xq, q, n_q, prm, &ref, form, precond, opts, &dref,
                               nullptr, stream));
    pb_quad_plan best = ref;
    double best_change = 0.0;
    auto change_of = [&](const pb_quad_plan& p, double* change) -> int {
        double d = 0.0;
        PB_TRY(pb_solvation_energy(ctx, verts, n_verts, tris, n_tris, xq, q, n_q, prm, &p, form, precond, opts, &d,
                                   nullptr, stream));
        *change = std::fabs(d / dref - 1.0);
        return PB_OK;
    };
    if (ref.far_q > 3 && ref.band_eta == 0.0) {
        const double etas[4] = {2.0, 3.0, 4.0, 6.0};
        for (double eta : etas) {
            pb_quad_plan p = ref;
            p.far_q = 3;
            p.band_eta = eta;
            p.band_q = ref.far_q;
            double change = 0.0;
            PB_TRY(change_of(p, &change));
            if (change <= tol_dG) {
                best = p;
                best_change = change;
                break;
            }
        }
    }
    // vertex, edge, coincident
    int* bcls[3] = {&best.n_ss_vert, &best.n_ss_edge, &best.n_ss_coin};
    for (int c = 0; c < 3; ++c) {
        if (*bcls[c] <= 1) continue;
        pb_quad_plan p = best;
        int* pc = c == 0 ? &p.n_ss_vert : c == 1 ? &p.n_ss_edge : &p.n_ss_coin;
        *pc -= 1;
        double change = 0.0;
        PB_TRY(change_of(p, &change));
        if (change <= tol_dG) {
            best = p;
            best_change = change;
        }
    }
    *out_plan = best;
    if (out_change) *out_change = best_change;
    return PB_OK;
}
