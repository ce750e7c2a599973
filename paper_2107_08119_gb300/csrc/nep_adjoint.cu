// nep_adjoint.cu -- gradient of the force loss with respect to the network
// parameters, by a hand-written adjoint of the force path.
//
// The paper fits without gradients (SNES, Sec. II.D); this is the
// differentiable route to the same force term of the loss.  With residuals
// e_i = F_i - F_tar_i over the N atoms of the training set and
// L_f = sqrt(sum_i |e_i|^2 / (3N)) (Eq. 30), and F_i = sum_j (dU_i/dr_ij -
// dU_j/dr_ji) (Eqs. 4-5):
//   dL_f/dz = sum_i sum_j d/dz(dU_i/dr_ij) . (delta_i - delta_j),
//   delta_i = e_i / (3N L_f).
// dU_i/dr_ij = sum_nu G_i,nu dq_i,nu/dr_ij (Eq. 23) and q does not depend on
// z, so
//   dL_f/dz = sum_i sum_nu dG_i,nu/dz lambda_i,nu,
//   lambda_i,nu = sum_j dq_i,nu/dr_ij . (delta_i - delta_j).
// For the network of Eqs. 21-22, G_nu = sum_mu w2_mu (1 - x_mu^2) w1_mu,nu;
// with s_mu = sum_nu w1_mu,nu lambda_nu and t_mu = 1 - x_mu^2, per atom:
//   d/dw2_mu    t_mu s_mu
//   d/db1_mu    2 w2_mu x_mu t_mu s_mu
//   d/dw1_mu,k  w2_mu t_mu lambda_k - 2 w2_mu x_mu t_mu s_mu q_k
//   d/db2       0
// The angular pair derivative follows the harmonic form of the force path:
// dq_nl/dr . d = sum_m 2 c_lm S_nlm (g_n' Z_lm (rhat . d) + g_n grad_u Z_lm . d_t),
// d_t = (d - (rhat . d) rhat) / r.
//
// Both passes recompute descriptors and pair derivatives from the positions;
// the only per-pair array is the forward's partial forces, which define F.
// Kernels (thread per atom, 128 per block, parameters in shared memory):
//   k_adj_site    q, network, dU_i/dr_ij for every CSR pair of the atom
//   k_adj_force   F_i = sum_p (pf[p] - pf[rev[p]]), e_i, block sums of |e|^2
//   k_adj_loss    L_f from the block sums (one block, fixed order)
//   k_adj_lambda  q and S again, lambda_i, the network terms; the block sums
//                 every parameter's terms over its atoms (FP32 in runs of 32
//                 atoms, FP64 across runs)
//   k_adj_grad    per parameter, the block sums in a fixed order
// Every sum has a fixed order: the gradient is bitwise reproducible.
#include <cmath>

#include "nep_dataset.cuh"

namespace nep {
namespace {

constexpr int kAdjThreads = 128;

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

// floats per atom row of the backward's block reduction: lambda[32], q[32],
// then a, c, t*s per neuron; odd so a warp writing one column of its rows
// hits 32 different banks
__host__ __device__ __forceinline__ int adj_row_stride(int nn) { return (kNdes * 2 + 3 * nn) | 1; }

__host__ __device__ __forceinline__ int pad32(int v) { return (v + 31) / 32 * 32; }

__device__ __forceinline__ void load_params(const float* __restrict__ z, int n_par, float* s_w)
{
    for (int t = threadIdx.x; t < n_par; t += blockDim.x) s_w[t] = z[t];
    __syncthreads();
}

__global__ void __launch_bounds__(kAdjThreads) k_adj_site(int N, const int* __restrict__ sid,
                                                          const Box* __restrict__ boxes,
                                                          const float* __restrict__ xh, const float* __restrict__ xl,
                                                          const long long* __restrict__ pstart,
                                                          const int* __restrict__ pj, const float* __restrict__ z,
                                                          int n_par, SiteParams P, float* __restrict__ pf,
                                                          unsigned* err)
{
    extern __shared__ float s_w[];
    load_params(z, n_par, s_w);
    P.w = s_w;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < N;
    const int ia = active ? i : 0;
    const long long p0 = pstart[ia];
    const int cnt = active ? (int)(pstart[ia + 1] - p0) : 0;
    const Box box = boxes[sid[ia]];
    const SlotTable T{pj + p0, 1, 0};
    const PfOut out{pf + 3 * p0, 3, 1};
    float uh, ul;
    site_partial_forces(ia, active, N, cnt, T, xh, xl, box, P, out, uh, ul);
    if (active && !isfinite(uh)) atomicOr(err, kErrNonFinite);
}

__global__ void __launch_bounds__(kAdjThreads) k_adj_force(int N, const long long* __restrict__ pstart,
                                                           const long long* __restrict__ rev,
                                                           const float* __restrict__ pf,
                                                           const float* __restrict__ f_tar, float4* __restrict__ res,
                                                           double* __restrict__ part, unsigned* err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double sq[1] = {0.0};
    if (i < N) {
        float F[3] = {0.f, 0.f, 0.f};
        for (long long p = pstart[i]; p < pstart[i + 1]; ++p) {
            const long long r = rev[p];
#pragma unroll
            for (int c = 0; c < 3; ++c) F[c] += pf[3 * p + c] - pf[3 * r + c];
        }
        const float ex = F[0] - f_tar[(size_t)3 * i], ey = F[1] - f_tar[(size_t)3 * i + 1],
                    ez = F[2] - f_tar[(size_t)3 * i + 2];
        res[i] = make_float4(ex, ey, ez, 0.f);
        if (!(isfinite(ex) && isfinite(ey) && isfinite(ez))) atomicOr(err, kErrNonFinite);
        sq[0] = (double)ex * ex + (double)ey * ey + (double)ez * ez;
    }
    block_sum_store<1>(sq, part + blockIdx.x);
}

// sums[0] = sum |e|^2, sums[1] = L_f; loss (optional) = L_f.
__global__ void k_adj_loss(int nblocks, int N, const double* __restrict__ part, double* __restrict__ sums,
                           double* __restrict__ loss)
{
    double v[1] = {0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v[0] += part[b];
    __shared__ double tot;
    block_sum_store<1>(v, &tot);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double L = sqrt(tot / (3.0 * (double)N));
        sums[0] = tot;
        sums[1] = L;
        if (loss) loss[0] = L;
    }
}

// One harmonic's share of lambda for a pair: with alpha = Z (rhat . d) and
// beta = grad_u Z . d_t, lambda_nl += A_nlm (g_n' alpha + g_n beta).
__device__ __forceinline__ void adj_term(const Harm& A, const float (&g)[kNA], const float (&dg)[kNA],
                                         int lm, float Y, float gx, float gy, float gz, float e, float tx, float ty,
                                         float tz, float (&lam)[kNdes])
{
    const float alpha = Y * e;
    const float beta = fmaf(gx, tx, fmaf(gy, ty, gz * tz));
#pragma unroll
    for (int n = 0; n < kNA; ++n)
        lam[kNR + n * kLmax + sh_l(lm)] = fmaf(harm(A, n, lm), fmaf(dg[n], alpha, g[n] * beta),
                                               lam[kNR + n * kLmax + sh_l(lm)]);
}

__device__ __forceinline__ void adj_pass(float x, float y, float z, const Harm& A, const float (&g)[kNA],
                                         const float (&dg)[kNA], float e, float tx, float ty, float tz,
                                         float (&lam)[kNdes])
{
    NEP_SH_LOCALS_FAST(x, y, z)
#define NEP_T(lm, Yv, gx, gy, gz) adj_term(A, g, dg, lm, Yv, gx, gy, gz, e, tx, ty, tz, lam);
    NEP_SH_TABLE(NEP_T)
#undef NEP_T
}

__global__ void __launch_bounds__(kAdjThreads) k_adj_lambda(int N, const int* __restrict__ sid,
                                                            const Box* __restrict__ boxes,
                                                            const float* __restrict__ xh,
                                                            const float* __restrict__ xl,
                                                            const long long* __restrict__ pstart,
                                                            const int* __restrict__ pj,
                                                            const float4* __restrict__ res,
                                                            const double* __restrict__ sums,
                                                            const float* __restrict__ z, int n_par, SiteParams P,
                                                            double* __restrict__ part)
{
    extern __shared__ float sm[];
    float* s_w = sm;
    const int nn = P.n_neu;
    const int stride = adj_row_stride(nn);
    float* rows = sm + pad32(n_par);
    load_params(z, n_par, s_w);
    P.w = s_w;
    float* row = rows + threadIdx.x * stride;

    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < N;
    const int ia = active ? i : 0;
    const long long p0 = pstart[ia];
    const int cnt = active ? (int)(pstart[ia + 1] - p0) : 0;
    const Box box = boxes[sid[ia]];
    const SlotTable T{pj + p0, 1, 0};
    const double L = sums[1];
    const float scale = L > 0.0 ? (float)(1.0 / (3.0 * (double)N * L)) : 0.f;

    float hi[3], li[3];
    load_pos(xh, xl, N, ia, hi, li);
    const float zi = load_z(xh, ia);
    float lam[kNdes];
    {
        float q[kNdes];
        Harm S;
        site_descriptors(ia, N, cnt, T, xh, xl, box, P, hi, li, zi, q, S);
#pragma unroll
        for (int v = 0; v < kNdes; ++v) row[kNdes + v] = q[v];
        // A_nlm = 2 c_lm S_nlm
#pragma unroll
        for (int a = 0; a < kNA; ++a)
#pragma unroll
            for (int m = 0; m < kLM; ++m) harm(S, a, m) *= 2.f * sh_c(m);
#pragma unroll
        for (int v = 0; v < kNdes; ++v) lam[v] = 0.f;
        const float4 ei = res[ia];
        const float di[3] = {ei.x * scale, ei.y * scale, ei.z * scale};
        for (int k = 0; k < cnt; ++k) {
            const int v = pj[p0 + k];
            const int j = v & 0xFFFFFF;
            float hj[3], lj[3];
            load_pos(xh, xl, N, j, hj, lj);
            const float4 ej = res[j];
            float r[3];
            pair_vector(ia, j, v >> 24, hi, li, hj, lj, box, r[0], r[1], r[2]);
            const float d2 = fmaf(r[0], r[0], fmaf(r[1], r[1], r[2] * r[2]));
            const float dd[3] = {fmaf(-ej.x, scale, di[0]), fmaf(-ej.y, scale, di[1]), fmaf(-ej.z, scale, di[2])};
            const float d = sqrtf(d2);
            const float inv = 1.f / d;
            const float u[3] = {r[0] * inv, r[1] * inv, r[2] * inv};
            const float e = fmaf(u[0], dd[0], fmaf(u[1], dd[1], u[2] * dd[2]));
            const float wz = pair_weight(P, zi, load_z(xh, j));
            if (d2 < P.rcR2) {
                float g[kNR], dg[kNR];
                radial_g_dg<kNR>(d, P.rcR, P.inv_rcR, g, dg, wz);
#pragma unroll
                for (int a = 0; a < kNR; ++a) lam[a] = fmaf(dg[a], e, lam[a]);
            }
            if (d2 < P.rcA2) {
                float g[kNA], dg[kNA];
                radial_g_dg<kNA>(d, P.rcA, P.inv_rcA, g, dg, wz);
                const float tx = fmaf(-e, u[0], dd[0]) * inv, ty = fmaf(-e, u[1], dd[1]) * inv,
                            tz = fmaf(-e, u[2], dd[2]) * inv;
                adj_pass(u[0], u[1], u[2], S, g, dg, e, tx, ty, tz, lam);
            }
        }
    }
#pragma unroll
    for (int v = 0; v < kNdes; ++v) row[v] = active ? lam[v] : 0.f;

    // network terms: x_mu again from q (row), s_mu = w1_mu . lambda
    const float* b1 = s_w + nn * kNdes;
    const float* w2 = b1 + nn;
    for (int mu = 0; mu < nn; ++mu) {
        const float* w = s_w + mu * kNdes;
        float a = -b1[mu], s = 0.f;
#pragma unroll
        for (int v = 0; v < kNdes; ++v) {
            a = fmaf(w[v], row[kNdes + v], a);
            s = fmaf(w[v], lam[v], s);
        }
        const float x = tanhf(a);
        const float t = fmaf(-x, x, 1.f);
        const float ts = active ? t * s : 0.f;
        row[2 * kNdes + mu] = active ? w2[mu] * t : 0.f;             // multiplies lambda_k in d/dw1
        row[2 * kNdes + nn + mu] = -2.f * w2[mu] * x * ts;            // multiplies q_k in d/dw1; -d/db1
        row[2 * kNdes + 2 * nn + mu] = ts;                            // d/dw2
    }
    if (!active)
#pragma unroll
        for (int v = 0; v < kNdes; ++v) row[kNdes + v] = 0.f;
    __syncthreads();

    // block sums of every parameter's per-atom terms
    const int nw1 = nn * kNdes;
    for (int o = threadIdx.x; o < n_par; o += blockDim.x) {
        double acc = 0.0;
        if (o < n_par - 1) {
            for (int r0 = 0; r0 < kAdjThreads; r0 += 32) {
                float s = 0.f;
                if (o < nw1) {
                    const int mu = o / kNdes, k = o % kNdes;
                    for (int r = r0; r < r0 + 32; ++r) {
                        const float* R = rows + r * stride;
                        s = fmaf(R[2 * kNdes + mu], R[k], fmaf(R[2 * kNdes + nn + mu], R[kNdes + k], s));
                    }
                } else if (o < nw1 + nn) {
                    const int mu = o - nw1;
                    for (int r = r0; r < r0 + 32; ++r) s -= rows[r * stride + 2 * kNdes + nn + mu];
                } else {
                    const int mu = o - nw1 - nn;
                    for (int r = r0; r < r0 + 32; ++r) s += rows[r * stride + 2 * kNdes + 2 * nn + mu];
                }
                acc += (double)s;
            }
        }
        part[(size_t)blockIdx.x * n_par + o] = acc;
    }
}

__global__ void k_adj_grad(int nblocks, int n_par, const double* __restrict__ part, const double* __restrict__ seed,
                           double* __restrict__ grad)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n_par) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * n_par + o];
    grad[o] = seed ? s * seed[0] : s;
}

template <class T>
int adj_alloc(T** p, size_t count)
{
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        return NEP_ERR_OOM;
    }
    return NEP_OK;
}

int ensure_adjoint(nep_model* m, nep_dataset* ds)
{
    AdjointScratch& a = ds->adj;
    if (a.pf) return NEP_OK;
    const int nb = blocks_for(ds->N, kAdjThreads);
    int rc;
    if ((rc = adj_alloc(&a.pf, (size_t)3 * ds->n_pairs)) || (rc = adj_alloc(&a.res, (size_t)4 * ds->N)) ||
        (rc = adj_alloc(&a.z, (size_t)m->n_par)) || (rc = adj_alloc(&a.part, (size_t)nb * m->n_par)) ||
        (rc = adj_alloc(&a.sums, 2))) {
        free_adjoint(a);
        return rc;
    }
    a.n_blocks = nb;
    a.ready = false;
    return NEP_OK;
}

SiteParams site_params(const nep_model* m, int typed)
{
    SiteParams P;
    P.typed = typed;
    P.w = nullptr;
    P.n_neu = m->hp.n_neu;
    P.rcR = (float)m->hp.rc_R;
    P.rcA = (float)m->hp.rc_A;
    P.rcR2 = P.rcR * P.rcR;
    P.rcA2 = P.rcA * P.rcA;
    P.inv_rcR = 1.f / P.rcR;
    P.inv_rcA = 1.f / P.rcA;
    return P;
}

}  // namespace

void free_adjoint(AdjointScratch& a)
{
    if (a.pf) cudaFree(a.pf);
    if (a.res) cudaFree(a.res);
    if (a.z) cudaFree(a.z);
    if (a.part) cudaFree(a.part);
    if (a.sums) cudaFree(a.sums);
    a = AdjointScratch();
}

}  // namespace nep

using namespace nep;

extern "C" {

int nep_force_loss(nep_model* m, nep_dataset* ds, const float* z, double* loss_f, void* stream)
{
    if (!m || !ds || ds->m != m || !z) {
        set_error("nep_force_loss: NULL argument or dataset of another model");
        return NEP_ERR_ARG;
    }
    int rc = ensure_adjoint(m, ds);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    AdjointScratch& a = ds->adj;
    const int N = ds->N, n_par = m->n_par, nb = a.n_blocks;
    rc = cuda_fail(cudaMemcpyAsync(a.z, z, sizeof(float) * n_par, cudaMemcpyDeviceToDevice, st),
                   "nep_force_loss: parameter copy");
    if (rc) return rc;
    const size_t smem = (size_t)pad32(n_par) * sizeof(float);
    k_adj_site<<<nb, kAdjThreads, smem, st>>>(N, ds->sid, ds->boxes, ds->xh, ds->xl, ds->pstart, ds->pj, a.z, n_par,
                                              site_params(m, ds->typed), a.pf, m->d_err);
    k_adj_force<<<nb, kAdjThreads, 0, st>>>(N, ds->pstart, ds->rev, a.pf, ds->f_tar, reinterpret_cast<float4*>(a.res),
                                            a.part, m->d_err);
    k_adj_loss<<<1, 256, 0, st>>>(nb, N, a.part, a.sums, loss_f);
    rc = cuda_fail(cudaGetLastError(), "force-loss forward kernels");
    if (rc) return rc;
    a.ready = true;
    return NEP_OK;
}

int nep_force_loss_backward(nep_model* m, nep_dataset* ds, const double* seed, double* grad, void* stream)
{
    if (!m || !ds || ds->m != m || !grad) {
        set_error("nep_force_loss_backward: NULL argument or dataset of another model");
        return NEP_ERR_ARG;
    }
    if (!ds->adj.ready) {
        set_error("nep_force_loss_backward: no nep_force_loss on this dataset before it");
        return NEP_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    AdjointScratch& a = ds->adj;
    const int N = ds->N, n_par = m->n_par, nb = a.n_blocks;
    const size_t smem = ((size_t)pad32(n_par) + (size_t)kAdjThreads * adj_row_stride(m->hp.n_neu)) * sizeof(float);
    int rc = cuda_fail(cudaFuncSetAttribute(k_adj_lambda, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                       "adjoint kernel shared memory");
    if (rc) return rc;
    k_adj_lambda<<<nb, kAdjThreads, smem, st>>>(N, ds->sid, ds->boxes, ds->xh, ds->xl, ds->pstart, ds->pj,
                                                reinterpret_cast<const float4*>(a.res), a.sums, a.z, n_par,
                                                site_params(m, ds->typed), a.part);
    k_adj_grad<<<blocks_for(n_par, 256), 256, 0, st>>>(nb, n_par, a.part, seed, grad);
    return cuda_fail(cudaGetLastError(), "force-loss adjoint kernels");
}

}  // extern "C"
