// nep_plain.cu -- the plain FP32 GPU form of the force path: the comparator
// the optimised path is measured against.
//
// One thread per atom, three unfused passes, no compensated sums:
//   k_plain_desc  q_n (Eq. 12) and q_nl by the literal O(M^2) double sum of
//                 Eq. 13 over neighbour pairs (j, k), k = j included, with
//                 Legendre polynomials P_l(cos theta_ijk)
//   k_plain_net   the network of Eqs. 21-22 and G = dU/dq
//   k_plain_pf    partial forces by Eqs. 23-25 (again O(M^2) per atom)
// and then the same assembly and reductions as the optimised path.  The
// neighbour list is shared with it.
#include <cmath>

#include "nep_internal.cuh"

namespace nep {
namespace {

constexpr int kPlainThreads = 128;
constexpr int kPlainMaxAng = 96;  // angular neighbours per atom held in local memory

__device__ __forceinline__ void plain_radial(float d, float rc, int nmax, float* g, float* dg)
{
    const float pi = 3.14159265358979f;
    const float x = 2.f * (d / rc - 1.f) * (d / rc - 1.f) - 1.f;
    const float dx = 4.f * (d / rc - 1.f) / rc;
    const float fc = 0.5f * (1.f + cosf(pi * d / rc));
    const float dfc = -0.5f * pi / rc * sinf(pi * d / rc);
    // T_n and dT_n/dx = n U_{n-1} by the recurrences of App. A
    float Tm = 1.f, Tc = x;        // T_{n-2}, T_{n-1} at order n >= 2
    float Um = 1.f, Uc = 2.f * x;  // U_{n-2}, U_{n-1} at order n >= 2
    for (int n = 0; n < nmax; ++n) {
        float T, dT;
        if (n == 0) {
            T = 1.f;
            dT = 0.f;
        } else if (n == 1) {
            T = x;
            dT = 1.f;
        } else {
            T = 2.f * x * Tc - Tm;
            Tm = Tc;
            Tc = T;
            dT = n * Uc;
            const float Un = 2.f * x * Uc - Um;
            Um = Uc;
            Uc = Un;
        }
        g[n] = 0.5f * (T + 1.f) * fc;
        if (dg) dg[n] = 0.5f * dT * dx * fc + 0.5f * (T + 1.f) * dfc;
    }
}

// P_l(c) and dP_l/dc for l = 1..4 (closed forms)
__device__ __forceinline__ void plain_legendre(float c, float (&P)[kLmax], float (&dP)[kLmax])
{
    const float c2 = c * c;
    P[0] = c;
    dP[0] = 1.f;
    P[1] = 1.5f * c2 - 0.5f;
    dP[1] = 3.f * c;
    P[2] = 2.5f * c2 * c - 1.5f * c;
    dP[2] = 7.5f * c2 - 1.5f;
    P[3] = 4.375f * c2 * c2 - 3.75f * c2 + 0.375f;
    dP[3] = 17.5f * c2 * c - 7.5f * c;
}

struct Gathered {
    int cnt;
    float u[kPlainMaxAng][3];
    float r[kPlainMaxAng];
    float g[kPlainMaxAng][kNA];
    float dg[kPlainMaxAng][kNA];
    int slot[kPlainMaxAng];
};

// Pair vector of slot k of atom i (list layout nbr[k][n]).
__device__ __forceinline__ float plain_pair(int i, int n, int k, const int* __restrict__ nbr,
                                            const float* __restrict__ xh, const float* __restrict__ xl,
                                            const Box& box, const float (&hi)[3], const float (&li)[3], float (&r)[3])
{
    const int v = nbr[(size_t)k * n + i];
    const int j = v & 0xFFFFFF;
    float hj[3], lj[3];
    load_pos(xh, xl, n, j, hj, lj);
    pair_vector(i, j, v >> 24, hi, li, hj, lj, box, r[0], r[1], r[2]);
    return r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
}

__device__ bool gather_angular(int i, int n, int cnt, const int* __restrict__ nbr, const float* __restrict__ xh,
                               const float* __restrict__ xl, const Box& box, float rcA, Gathered& A)
{
    float hi[3], li[3];
    load_pos(xh, xl, n, i, hi, li);
    A.cnt = 0;
    for (int k = 0; k < cnt; ++k) {
        float r[3];
        const float d2 = plain_pair(i, n, k, nbr, xh, xl, box, hi, li, r);
        if (!(d2 < rcA * rcA)) continue;
        if (A.cnt >= kPlainMaxAng) return false;
        const float d = sqrtf(d2);
        const int a = A.cnt++;
        A.r[a] = d;
        A.slot[a] = k;
        for (int c = 0; c < 3; ++c) A.u[a][c] = r[c] / d;
        plain_radial(d, rcA, kNA, A.g[a], A.dg[a]);
    }
    return true;
}

__global__ void __launch_bounds__(kPlainThreads) k_plain_desc(int n, int m_cap, const int* __restrict__ count,
                                                              const int* __restrict__ nbr,
                                                              const float* __restrict__ xh,
                                                              const float* __restrict__ xl, Box box, float rcR,
                                                              float rcA, float* __restrict__ q, unsigned* err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int cnt = min(count[i], m_cap);
    float hi[3], li[3];
    load_pos(xh, xl, n, i, hi, li);
    float qd[kNdes];
    for (int v = 0; v < kNdes; ++v) qd[v] = 0.f;
    for (int k = 0; k < cnt; ++k) {
        float r[3];
        const float d2 = plain_pair(i, n, k, nbr, xh, xl, box, hi, li, r);
        if (!(d2 < rcR * rcR)) continue;
        float g[kNR];
        plain_radial(sqrtf(d2), rcR, kNR, g, nullptr);
        for (int a = 0; a < kNR; ++a) qd[a] += g[a];
    }
    Gathered A;
    if (!gather_angular(i, n, cnt, nbr, xh, xl, box, rcA, A)) {
        atomicOr(err, kErrOverflow);
        return;
    }
    for (int a = 0; a < A.cnt; ++a)
        for (int b = 0; b < A.cnt; ++b) {
            const float c = A.u[a][0] * A.u[b][0] + A.u[a][1] * A.u[b][1] + A.u[a][2] * A.u[b][2];
            float P[kLmax], dP[kLmax];
            plain_legendre(c, P, dP);
            for (int nn = 0; nn < kNA; ++nn) {
                const float gg = A.g[a][nn] * A.g[b][nn];
                for (int l = 0; l < kLmax; ++l) qd[kNR + nn * kLmax + l] += gg * P[l];
            }
        }
    for (int v = 0; v < kNdes; ++v) q[(size_t)v * n + i] = qd[v];
}

__global__ void __launch_bounds__(kPlainThreads) k_plain_net(int n, int n_neu, const float* __restrict__ z,
                                                             const float* __restrict__ q, float* __restrict__ G,
                                                             double* __restrict__ e_atom, double* __restrict__ e_part,
                                                             unsigned* err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double e[1] = {0.0};
    if (i < n) {
        const float* b1 = z + n_neu * kNdes;
        const float* w2 = b1 + n_neu;
        float qv[kNdes], g[kNdes];
        for (int v = 0; v < kNdes; ++v) {
            qv[v] = q[(size_t)v * n + i];
            g[v] = 0.f;
        }
        float U = -w2[n_neu];
        for (int mu = 0; mu < n_neu; ++mu) {
            float a = -b1[mu];
            for (int v = 0; v < kNdes; ++v) a += z[mu * kNdes + v] * qv[v];
            const float x = tanhf(a);
            U += w2[mu] * x;
            const float d = w2[mu] * (1.f - x * x);
            for (int v = 0; v < kNdes; ++v) g[v] += d * z[mu * kNdes + v];
        }
        for (int v = 0; v < kNdes; ++v) G[(size_t)v * n + i] = g[v];
        if (e_atom) e_atom[i] = U;
        if (!isfinite(U)) atomicOr(err, kErrNonFinite);
        e[0] = U;
    }
    block_sum_store<1>(e, e_part + blockIdx.x);
}

__global__ void __launch_bounds__(kPlainThreads) k_plain_pf(int n, int m_cap, const int* __restrict__ count,
                                                            const int* __restrict__ nbr, const float* __restrict__ xh,
                                                            const float* __restrict__ xl, Box box, float rcR,
                                                            float rcA, const float* __restrict__ G,
                                                            float* __restrict__ pf, unsigned* err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int cnt = min(count[i], m_cap);
    float Gv[kNdes];
    for (int v = 0; v < kNdes; ++v) Gv[v] = G[(size_t)v * n + i];
    float hi[3], li[3];
    load_pos(xh, xl, n, i, hi, li);
    const float rc2 = fmaxf(rcR * rcR, rcA * rcA);
    // radial part for every slot (zero partial force outside both cutoffs is not stored)
    for (int k = 0; k < cnt; ++k) {
        float r[3];
        const float d2 = plain_pair(i, n, k, nbr, xh, xl, box, hi, li, r);
        if (!(d2 < rc2)) continue;
        float p[3] = {0.f, 0.f, 0.f};
        if (d2 < rcR * rcR) {
            const float d = sqrtf(d2);
            float g[kNR], dg[kNR];
            plain_radial(d, rcR, kNR, g, dg);
            float s = 0.f;
            for (int a = 0; a < kNR; ++a) s += Gv[a] * dg[a];
            for (int c = 0; c < 3; ++c) p[c] = s * r[c] / d;
        }
        float* o = pf + 4 * ((size_t)k * n + i);  // pf[k][i] float4 record
        for (int c = 0; c < 3; ++c) o[c] = p[c];
    }
    Gathered A;
    if (!gather_angular(i, n, cnt, nbr, xh, xl, box, rcA, A)) {
        atomicOr(err, kErrOverflow);
        return;
    }
    // angular part: dq_nl/dr_ij = 2 sum_k [g_n'(r_ij) g_n(r_ik) P_l u_j
    //                                      + g_n(r_ij) g_n(r_ik) P_l' (u_k - c u_j) / r_ij]
    for (int a = 0; a < A.cnt; ++a) {
        float p[3] = {0.f, 0.f, 0.f};
        for (int b = 0; b < A.cnt; ++b) {
            const float c = A.u[a][0] * A.u[b][0] + A.u[a][1] * A.u[b][1] + A.u[a][2] * A.u[b][2];
            float P[kLmax], dP[kLmax];
            plain_legendre(c, P, dP);
            float s1 = 0.f, s2 = 0.f;
            for (int nn = 0; nn < kNA; ++nn)
                for (int l = 0; l < kLmax; ++l) {
                    const float Gl = Gv[kNR + nn * kLmax + l];
                    s1 += Gl * A.dg[a][nn] * A.g[b][nn] * P[l];
                    s2 += Gl * A.g[a][nn] * A.g[b][nn] * dP[l];
                }
            for (int cc = 0; cc < 3; ++cc)
                p[cc] += 2.f * (s1 * A.u[a][cc] + s2 * (A.u[b][cc] - c * A.u[a][cc]) / A.r[a]);
        }
        float* o = pf + 4 * ((size_t)A.slot[a] * n + i);
        for (int cc = 0; cc < 3; ++cc) o[cc] += p[cc];
    }
}

}  // namespace

int launch_plain_site(const ForceArgs& a, NeighborList& nl, int n, float* q, float* G, double* e_atom,
                      double* e_partials, unsigned* d_err, cudaStream_t st, int& nblocks)
{
    nl.mask_set = false;  // the assembly tests every slot's distance itself
    nblocks = (n + kPlainThreads - 1) / kPlainThreads;
    k_plain_desc<<<nblocks, kPlainThreads, 0, st>>>(n, nl.m_cap, nl.count, nl.nbr, nl.xh, nl.xl, a.box, a.rcR, a.rcA,
                                                    q, d_err);
    k_plain_net<<<nblocks, kPlainThreads, 0, st>>>(n, a.n_neu, a.z, q, G, e_atom, e_partials, d_err);
    k_plain_pf<<<nblocks, kPlainThreads, 0, st>>>(n, nl.m_cap, nl.count, nl.nbr, nl.xh, nl.xl, a.box, a.rcR, a.rcA,
                                                  G, nl.pf, d_err);
    return cuda_fail(cudaGetLastError(), "plain force kernels");
}

}  // namespace nep
