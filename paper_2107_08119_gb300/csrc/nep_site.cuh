// nep_site.cuh -- per-atom NEP arithmetic of the force path, in FP32.
//
// For one atom i with Verlet-list slots k:
//   radial descriptors   q_n = sum_j g_n(r_ij)                     (Eq. 12)
//   angular descriptors  q_nl = sum_{j,k} g_n g_n P_l(cos theta)   (Eq. 13)
//     evaluated exactly through the addition theorem (Eqs. 17-18 with
//     n = n'): P_l(u.v) = sum_m c_lm Z_lm(u) Z_lm(v) for the real solid
//     harmonics Z_lm below, so q_nl = sum_m c_lm S_nlm^2 with
//     S_nlm = sum_j g_n(r_ij) Z_lm(rhat_ij): O(M) instead of O(M^2);
//   g_n = (T_n(x) + 1)/2 f_c(r), x = 2 (r/r_c - 1)^2 - 1            (Eq. 14)
//   f_c = (1 + cos(pi r / r_c))/2                                  (Eq. 15)
//   network  x_mu = tanh(sum_nu w1 q - b1), U = sum_mu w2 x - b2     (Eqs. 21-22)
//   G_nu = dU/dq_nu = sum_mu w2_mu (1 - x_mu^2) w1_mu,nu
//   partial force dU_i/dr_ij = sum_nu G_nu dq_nu/dr_ij               (Eqs. 23-25)
//     radial: G_n g_n'(r) rhat; angular: sum_nlm 2 c_lm G_nl S_nlm grad(g_n Z_lm),
//     grad(g Z(rhat)) = g' Z rhat + g (grad_u Z - rhat (rhat . grad_u Z)) / r.
// Chebyshev T_n and U_n come from the recurrences of App. A (Eqs. A1-A3).
//
// The functions are __host__ __device__ so the same code can be exercised
// on the CPU; on the device the weights pointer refers to shared memory.
#pragma once

#include <math.h>

#include "nep_internal.cuh"

namespace nep {

__host__ __device__ __forceinline__ void sincospi_f(float x, float* s, float* c)
{
#ifdef __CUDA_ARCH__
    sincospif(x, s, c);
#else
    *s = (float)sin(3.14159265358979323846 * (double)x);
    *c = (float)cos(3.14159265358979323846 * (double)x);
#endif
}

// d / rc from d * (1/rc) with one Newton correction: the rounded reciprocal
// of a cutoff such as 5 A is not exact in FP32, and the plain product would
// bias every radial function the same way.
__host__ __device__ __forceinline__ float div_rc(float d, float rc, float inv_rc)
{
    const float q0 = d * inv_rc;
    return fmaf(fmaf(-q0, rc, d), inv_rc, q0);
}

// Error-free sum: s + e == a + b exactly (Knuth's TwoSum).
__host__ __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// g_n(d), n = 0..N-1, for d < rc; w multiplies the cutoff function (the
// multicomponent weight sqrt(Z_i Z_j), 1 for one species).  x = 2 t^2 - 1
// with t = d/rc - 1 carried as hi + lo: for d < rc/2 the difference rounds,
// and the Chebyshev recurrence multiplies an error in x by up to n^2.
template <int N>
__host__ __device__ __forceinline__ void radial_g(float d, float rc, float inv_rc, float (&g)[N], float w = 1.f)
{
    float s, c;
    const float dr = div_rc(d, rc, inv_rc);
    sincospi_f(dr, &s, &c);
    const float fc = 0.5f * (1.f + c) * w;
    float t, tl;
    two_sum(dr, -1.f, t, tl);
    const float x = fmaf(4.f * t, tl, fmaf(2.f * t, t, -1.f));
    float Tm = 1.f, T = x;  // T_{n-1}, T_n
    const float hfc = 0.5f * fc;
    g[0] = fc;
    if (N > 1) g[1] = fmaf(hfc, x, hfc);
#pragma unroll
    for (int n = 2; n < N; ++n) {
        const float Tn = fmaf(2.f * x, T, -Tm);
        Tm = T;
        T = Tn;
        g[n] = fmaf(hfc, Tn, hfc);
    }
}

// (g_n(d), dg_n/dd), n = 0..N-1, for d < rc, as pairs; w as in radial_g.
template <int N>
__host__ __device__ __forceinline__ void radial_gd(float d, float rc, float inv_rc, float2 (&gd)[N], float w = 1.f)
{
    float s, c;
    const float dr = div_rc(d, rc, inv_rc);
    sincospi_f(dr, &s, &c);
    const float fc = 0.5f * (1.f + c) * w;
    const float dfc = -0.5f * 3.14159265358979f * inv_rc * s * w;
    const float t = dr - 1.f;
    const float x = fmaf(2.f * t, t, -1.f);
    const float dxdr = 4.f * t * inv_rc;
    const float hfc = 0.5f * fc, hdfc = 0.5f * dfc;
    const float a = hfc * dxdr;  // (1/2) f_c dx/dr
    float Tm = 1.f, T = x;       // T_{n-1}, T_n
    float Um = 1.f, U = 2.f * x; // U_{n-2}, U_{n-1} when at order n
    gd[0] = make_float2(fc, dfc);
    if (N > 1) gd[1] = make_float2(fmaf(hfc, x, hfc), fmaf(a, 1.f, fmaf(hdfc, x, hdfc)));  // dT_1/dx = U_0 = 1
#pragma unroll
    for (int n = 2; n < N; ++n) {
        const float Tn = fmaf(2.f * x, T, -Tm);
        Tm = T;
        T = Tn;
        // dT_n/dx = n U_{n-1}; U at this point holds U_{n-1}
        gd[n] = make_float2(fmaf(hfc, Tn, hfc), fmaf(a * (float)n, U, fmaf(hdfc, Tn, hdfc)));
        const float Un = fmaf(2.f * x, U, -Um);
        Um = U;
        U = Un;
    }
}

// g_n(d) and dg_n/dd, n = 0..N-1, for d < rc, as two arrays; w as in radial_g.
template <int N>
__host__ __device__ __forceinline__ void radial_g_dg(float d, float rc, float inv_rc, float (&g)[N], float (&dg)[N],
                                                     float w = 1.f)
{
    float2 gd[N];
    radial_gd<N>(d, rc, inv_rc, gd, w);
#pragma unroll
    for (int n = 0; n < N; ++n) {
        g[n] = gd[n].x;
        dg[n] = gd[n].y;
    }
}

// The 24 real solid-harmonic polynomials Z_lm(u) with 1 <= l <= 4 (u a unit
// vector), listed once as T(lm, Z, dZ/dux, dZ/duy, dZ/duz), and the
// addition-theorem weights c_lm with sum_m c_lm Z_lm(u) Z_lm(v) = P_l(u . v)
// (Eqs. 17-18: c_lm = 4 pi/(2l+1) times the squared normalisation of the
// real spherical harmonic).  Every c_lm is a dyadic rational, exact in FP32.
// The gradient columns are those of the polynomial extension off the sphere;
// callers project them onto the tangent plane.  Expects the locals of
// NEP_SH_LOCALS in scope; the factors k z^2 - c are formed from the exact
// square (the rounding of z^2 would otherwise be multiplied by up to 21).
#define NEP_SH_LOCALS(x, y, z)                                                  \
    const float x2 = x * x, y2 = y * y, z2 = z * z;                             \
    const float xy = x * y, yz = y * z, xz = x * z;                             \
    const float x2my2 = x2 - y2;                                                \
    const float z2l = fmaf(z, z, -z2); /* z^2 = z2 + z2l exactly */             \
    const float a5 = fmaf(5.f, z2l, fmaf(5.f, z2, -1.f));                       \
    const float a7 = fmaf(7.f, z2l, fmaf(7.f, z2, -1.f));                       \
    const float b7 = fmaf(7.f, z2l, fmaf(7.f, z2, -3.f));                       \
    const float c21 = fmaf(21.f, z2l, fmaf(21.f, z2, -3.f));                    \
    const float e19 = fmaf(35.f, z2l, fmaf(35.f, z2, -30.f));                   \
    (void)x2my2; (void)z2l; (void)a5; (void)a7; (void)b7; (void)c21; (void)e19;

// The same with z^2 rounded once (the partial forces, whose 1e-4 eV/A bar
// leaves room).
#define NEP_SH_LOCALS_FAST(x, y, z)                                                \
    const float x2 = x * x, y2 = y * y, z2 = z * z;                             \
    const float xy = x * y, yz = y * z, xz = x * z;                             \
    const float x2my2 = x2 - y2;                                                \
    const float z2l = 0.f;                                                      \
    const float a5 = 5.f * z2 - 1.f, a7 = 7.f * z2 - 1.f, b7 = 7.f * z2 - 3.f; \
    const float c21 = 21.f * z2 - 3.f, e19 = 35.f * z2 - 30.f;                  \
    (void)x2my2; (void)z2l; (void)a5; (void)a7; (void)b7; (void)c21; (void)e19;

#define NEP_SH_TABLE(T)                                                                             \
    /* l = 1 */                                                                                     \
    T(0, x, 1.f, 0.f, 0.f)                                                                          \
    T(1, y, 0.f, 1.f, 0.f)                                                                          \
    T(2, z, 0.f, 0.f, 1.f)                                                                          \
    /* l = 2 */                                                                                     \
    T(3, xy, y, x, 0.f)                                                                             \
    T(4, yz, 0.f, z, y)                                                                             \
    T(5, xz, z, 0.f, x)                                                                             \
    T(6, fmaf(3.f, z2l, fmaf(3.f, z2, -1.f)), 0.f, 0.f, 6.f * z)                                                         \
    T(7, x2my2, 2.f * x, -2.f * y, 0.f)                                                             \
    /* l = 3 */                                                                                     \
    T(8, y * (3.f * x2 - y2), 6.f * xy, 3.f * x2my2, 0.f)                                           \
    T(9, xy * z, yz, xz, xy)                                                                        \
    T(10, y * a5, 0.f, a5, 10.f * yz)                                                               \
    T(11, z * fmaf(5.f, z2l, fmaf(5.f, z2, -3.f)), 0.f, 0.f, 15.f * z2 - 3.f)                                          \
    T(12, x * a5, a5, 0.f, 10.f * xz)                                                               \
    T(13, z * x2my2, 2.f * xz, -2.f * yz, x2my2)                                                    \
    T(14, x * (x2 - 3.f * y2), 3.f * x2my2, -6.f * xy, 0.f)                                         \
    /* l = 4 */                                                                                     \
    T(15, xy * x2my2, y * (3.f * x2 - y2), x * (x2 - 3.f * y2), 0.f)                                \
    T(16, yz * (3.f * x2 - y2), 6.f * xy * z, 3.f * z * x2my2, y * (3.f * x2 - y2))                  \
    T(17, xy * a7, y * a7, x * a7, 14.f * xy * z)                                                   \
    T(18, yz * b7, 0.f, z * b7, y * c21)                                                            \
    T(19, fmaf(z2, e19, fmaf(z2l, e19, 3.f)), 0.f, 0.f, z * (140.f * z2 - 60.f))                         \
    T(20, xz * b7, z * b7, 0.f, x * c21)                                                            \
    T(21, x2my2 * a7, 2.f * x * a7, -2.f * y * a7, 14.f * z * x2my2)                                \
    T(22, xz * (x2 - 3.f * y2), 3.f * z * x2my2, -6.f * xy * z, x * (x2 - 3.f * y2))                 \
    T(23, x2 * (x2 - 3.f * y2) - y2 * (3.f * x2 - y2), 4.f * x * (x2 - 3.f * y2), 4.f * y * (y2 - 3.f * x2), 0.f)

// addition-theorem weights c_lm in the order of NEP_SH_TABLE
__host__ __device__ __forceinline__ constexpr float sh_c(int lm)
{
    constexpr float c[kLM] = {1.f,          1.f,          1.f,                                        // l = 1
                              3.f,          3.f,          3.f,          0.25f,        0.75f,        // l = 2
                              0.625f,       15.f,         0.375f,       0.25f,        0.375f,       // l = 3
                              3.75f,        0.625f,                                                 //
                              8.75f,        4.375f,       1.25f,        0.625f,       0.015625f,    // l = 4
                              0.625f,       0.3125f,      4.375f,       0.546875f};                 //
    return c[lm];
}

// l of harmonic index lm (0-based l - 1)
__host__ __device__ __forceinline__ constexpr int sh_l(int lm) { return lm < 3 ? 0 : (lm < 8 ? 1 : (lm < 15 ? 2 : 3)); }

// Descriptor sizes of a model: NR radial orders (n_max^R + 1), NA angular
// radial orders (n_max^A + 1), l = 1..4; N_des = NR + 4 NA (Eq. 16).  The
// site functions below are templates over these sizes: Desc<8, 6> is the
// 32-descriptor model of the Si workloads, Desc<13, 7> the 41-descriptor
// model with the split hyperparameters of the paper's PbTe potential.
template <int NR_, int NA_>
struct Desc {
    static constexpr int NR = NR_;
    static constexpr int NA = NA_;
    static constexpr int NA2 = (NA_ + 1) / 2;  // angular orders in pairs (odd NA: the last pair's y is unused)
    static constexpr int Ndes = NR_ + NA_ * kLmax;
};
using DescSi = Desc<kNR, kNA>;
using DescPbTe = Desc<13, 7>;
static_assert(DescSi::Ndes == kNdes, "the default model has 32 descriptors");
static_assert(DescPbTe::Ndes == 41, "the split model has 41 descriptors");

// Harmonic sums S_nlm of one atom (later the coefficients A_nlm), the radial
// orders in pairs (2p, 2p + 1) so that one packed f32x2 FMA updates two.
template <class D>
using HarmT = float2[D::NA2][kLM];
constexpr int kNA2 = DescSi::NA2;
typedef HarmT<DescSi> Harm;

template <int N2>
__host__ __device__ __forceinline__ float& harm(float2 (&S)[N2][kLM], int n, int lm)
{
    return (n & 1) ? S[n >> 1][lm].y : S[n >> 1][lm].x;
}
template <int N2>
__host__ __device__ __forceinline__ float harm(const float2 (&S)[N2][kLM], int n, int lm)
{
    return (n & 1) ? S[n >> 1][lm].y : S[n >> 1][lm].x;
}

// g_n paired as (g_2p, g_2p+1); an odd last order is paired with 0
template <int NA, int N2>
__host__ __device__ __forceinline__ void pair_orders(const float (&g)[NA], float2 (&g2)[N2])
{
    static_assert(N2 == (NA + 1) / 2, "paired orders");
#pragma unroll
    for (int p = 0; p < N2; ++p) g2[p] = make_float2(g[2 * p], 2 * p + 1 < NA ? g[2 * p + 1] : 0.f);
}

// S[n][lm] += g[n] * Y_lm(u), two radial orders per packed FMA
template <int N2>
__host__ __device__ __forceinline__ void sh_acc(float2 (&S)[N2][kLM], const float2 (&g2)[N2], int lm, float Y)
{
#pragma unroll
    for (int p = 0; p < N2; ++p) S[p][lm] = ffma2(g2[p], bcast2(Y), S[p][lm]);
}

template <int N2>
__host__ __device__ __forceinline__ void sh_pass1(float x, float y, float z, const float2 (&g)[N2],
                                                  float2 (&S)[N2][kLM])
{
    NEP_SH_LOCALS(x, y, z)
#define NEP_T(lm, Yv, gx, gy, gz) sh_acc(S, g, lm, Yv);
    NEP_SH_TABLE(NEP_T)
#undef NEP_T
}

// One harmonic's contribution to the angular partial force:
//   (cg, cd) = sum_n A[n][lm] (g_n, g_n')   (one packed FMA per order)
//   B += cd Y, V += cg grad_u Y             ((Vx, Vy) packed).
template <int NA, int N2>
__host__ __device__ __forceinline__ void sh_term(const float2 (&A)[N2][kLM], const float2 (&gd)[NA], int lm, float Y,
                                                 float gx, float gy, float gz, float& B, float2& Vxy, float& Vz)
{
    float2 c = make_float2(0.f, 0.f);
#pragma unroll
    for (int n = 0; n < NA; ++n) c = ffma2(bcast2(harm(A, n, lm)), gd[n], c);
    B = fmaf(c.y, Y, B);
    Vxy = ffma2(bcast2(c.x), make_float2(gx, gy), Vxy);
    Vz = fmaf(c.x, gz, Vz);
}

template <int NA, int N2>
__host__ __device__ __forceinline__ void sh_pass2(float x, float y, float z, const float2 (&A)[N2][kLM],
                                                  const float2 (&gd)[NA], float& B, float2& Vxy, float& Vz)
{
    NEP_SH_LOCALS_FAST(x, y, z)
#define NEP_T(lm, Yv, gx, gy, gz) sh_term(A, gd, lm, Yv, gx, gy, gz, B, Vxy, Vz);
    NEP_SH_TABLE(NEP_T)
#undef NEP_T
}

// All 24 harmonics and their (unprojected) gradients.
__host__ __device__ __forceinline__ void sh_eval(float x, float y, float z, float (&Y)[kLM], float (&dY)[kLM][3])
{
    NEP_SH_LOCALS_FAST(x, y, z)
#define NEP_T(lm, Yv, gx, gy, gz) \
    Y[lm] = Yv;                   \
    dY[lm][0] = gx;               \
    dY[lm][1] = gy;               \
    dY[lm][2] = gz;
    NEP_SH_TABLE(NEP_T)
#undef NEP_T
}

// One neuron's compensated (Kahan) pre-activation a - ca = sum_v row_v q_v - b1:
// the rounding of a plain FP32 dot product feeds straight into U for every
// unsaturated neuron.
__host__ __device__ __forceinline__ void kahan_step(float w, float qv, float& a, float& ca)
{
    const float y = fmaf(w, qv, -ca);
    const float t = a + y;
    ca = (t - a) - y;
    a = t;
}

// Adds neuron mu's output w2 x to the compensated sum (s, c) and its share
// w2 (1 - x^2) w1_mu of G.
template <int ND>
__host__ __device__ __forceinline__ void neuron_out(float w2, float xm, const float* row, float& s, float& c,
                                                    float (&G)[ND])
{
    const float p = w2 * xm;
    const float ep = fmaf(w2, xm, -p);
    float t, e;
    two_sum(s, p, t, e);
    s = t;
    c += e + ep;
    const float d = w2 * fmaf(-xm, xm, 1.f);
#ifdef __CUDA_ARCH__
    if constexpr (ND % 4 == 0) {
        // the row is 16-byte aligned (shared memory, ND floats per row)
        const float4* row4 = reinterpret_cast<const float4*>(row);
#pragma unroll
        for (int v = 0; v < ND; v += 4) {
            const float4 t = row4[v / 4];
            G[v] = fmaf(d, t.x, G[v]);
            G[v + 1] = fmaf(d, t.y, G[v + 1]);
            G[v + 2] = fmaf(d, t.z, G[v + 2]);
            G[v + 3] = fmaf(d, t.w, G[v + 3]);
        }
    } else
#endif
    {
#pragma unroll
        for (int v = 0; v < ND; ++v) G[v] = fmaf(d, row[v], G[v]);
    }
}

// Network of Eqs. 21-22 and its input gradient.  w points at the parameter
// vector [w1 (n_neu x N_des), b1, w2, b2].  The pre-activations and the output
// sum are compensated (rounding errors carried along) because the site energy
// must hold ~1e-7 relative accuracy.  Returns U as hi + lo.
template <int ND>
__host__ __device__ __forceinline__ void network(const float* w, int n_neu, const float (&q)[ND], float (&G)[ND],
                                                 float& U_hi, float& U_lo)
{
    const float* b1 = w + n_neu * ND;
    const float* w2 = b1 + n_neu;
    const float b2 = w2[n_neu];
#pragma unroll
    for (int v = 0; v < ND; ++v) G[v] = 0.f;
    float s = 0.f, c = 0.f;
    for (int mu = 0; mu < n_neu; ++mu) {
        const float* row = w + mu * ND;
        // four interleaved compensated chains (descriptor v in chain v mod 4),
        // so that consecutive steps do not wait on each other, joined by
        // error-free sums
        float a[4] = {-b1[mu], 0.f, 0.f, 0.f}, ca[4] = {0.f, 0.f, 0.f, 0.f};
#ifdef __CUDA_ARCH__
        if constexpr (ND % 4 == 0) {
            // 16-byte loads of the row (shared memory, aligned for ND % 4 == 0)
            const float4* row4 = reinterpret_cast<const float4*>(row);
#pragma unroll
            for (int v = 0; v < ND; v += 4) {
                const float4 t = row4[v / 4];
                kahan_step(t.x, q[v], a[0], ca[0]);
                kahan_step(t.y, q[v + 1], a[1], ca[1]);
                kahan_step(t.z, q[v + 2], a[2], ca[2]);
                kahan_step(t.w, q[v + 3], a[3], ca[3]);
            }
        } else
#endif
        {
#pragma unroll
            for (int v = 0; v < ND; ++v) kahan_step(row[v], q[v], a[v & 3], ca[v & 3]);
        }
        float s01, e01, s23, e23, sa, ea;
        two_sum(a[0], a[1], s01, e01);
        two_sum(a[2], a[3], s23, e23);
        two_sum(s01, s23, sa, ea);
        const float comp = ((ca[0] + ca[1]) + (ca[2] + ca[3])) - ((e01 + e23) + ea);
        neuron_out(w2[mu], tanhf(sa - comp), row, s, c, G);
    }
    float t, e;
    two_sum(s, -b2, t, e);
    U_hi = t;
    U_lo = c + e;
}

// One neighbour slot: packed index and the neighbour's hi/lo position.  The
// loops below fetch slot k+1 (or k-1) before working on slot k so the loads
// overlap the arithmetic of the current slot.
struct NbSlot {
    int v;
    float h[3], l[3];
    float z;  // the neighbour's species number
};

// Slot k of the atom is slots[k * stride + idx]: the global list (stride n,
// idx i) or a block's staged copy in shared memory (stride blockDim, idx tid).
struct SlotTable {
    const int* slots;
    int stride;
    int idx;
    // for a compacted table (only the slots within the cutoff, in their
    // order): the original slot of entry k at orig[k * stride + idx]
    const unsigned char* orig = nullptr;
};

__host__ __device__ __forceinline__ void fetch_slot(const SlotTable& T, const float* __restrict__ xh,
                                                    const float* __restrict__ xl, int n, int k, int cnt, NbSlot& s)
{
    if (k >= 0 && k < cnt) {
        s.v = T.slots[(size_t)k * T.stride + T.idx];
        load_pos(xh, xl, n, s.v & 0xFFFFFF, s.h, s.l);
        s.z = load_z(xh, s.v & 0xFFFFFF);
    }
}

// Parameters of the per-atom site functions.
struct SiteParams {
    const float* w;  // parameters (shared memory on the device)
    int n_neu;
    float rcR, rcA, rcR2, rcA2, inv_rcR, inv_rcA;
    int typed;       // multicomponent weighting sqrt(Z_i Z_j) (0: one species, weight 1)
};

// the multicomponent weight of a pair (Sec. II.A): sqrt(Z_i Z_j), 1 for one species
__host__ __device__ __forceinline__ float pair_weight(const SiteParams& P, float zi, float zj)
{
    return P.typed ? sqrtf(zi * zj) : 1.f;
}

// Where the partial force of slot k goes: base[k * slot_stride + c * comp_stride].
// The MD list stores pf[k][c][i] (base = pf + i, strides 3n and n); a
// training-set CSR list stores pf[p][c] (base = pf + 3 p0, strides 3 and 1).
struct PfOut {
    float* base;
    size_t slot_stride;
    size_t comp_stride;
};

// Unit vector r / |r| with each component rounded once from a near-exact
// value.  The solid harmonics of degree l scale as |u|^l, so an error delta
// in the length of u enters every harmonic sum of that pair as l * delta: the
// plain r * (1 / sqrtf(d2)) is off in length by up to ~2.5 ulp, which
// carried into q_nl (Eq. 13) and the site energy at the 1e-6 eV level.  Here
// d2 is an unevaluated sum (exact squares, compensated additions), 1/|r| is
// one Newton step from the FP32 reciprocal square root evaluated in that
// precision and kept as hi + lo, and each component is r_a (hi + lo) with a
// single final rounding.
__host__ __device__ __forceinline__ void unit_vector(float rx, float ry, float rz, float& ux, float& uy, float& uz)
{
    const float px = rx * rx, py = ry * ry, pz = rz * rz;
    const float ex = fmaf(rx, rx, -px), ey = fmaf(ry, ry, -py), ez = fmaf(rz, rz, -pz);
    float s1, t1, sh, t2;
    two_sum(px, py, s1, t1);
    two_sum(s1, pz, sh, t2);
    const float sl = ((t1 + t2) + (ex + ey)) + ez;  // |r|^2 = sh + sl
    const float y0 = 1.f / sqrtf(sh);
    // residual 1 - |r|^2 y0^2, with sh * y0 * y0 split exactly into b + be + ae * y0
    const float a = sh * y0, ae = fmaf(sh, y0, -a);
    const float b = a * y0, be = fmaf(a, y0, -b);
    const float res = fmaf(-ae, y0, (1.f - b) - be) - sl * y0 * y0;
    const float yh = fmaf(0.5f * y0, res, y0);
    const float yl = fmaf(0.5f * y0, res, y0 - yh);  // 1/|r| = yh + yl
    const float qx = rx * yh, qy = ry * yh, qz = rz * yh;
    ux = qx + fmaf(rx, yl, fmaf(rx, yh, -qx));
    uy = qy + fmaf(ry, yl, fmaf(ry, yh, -qy));
    uz = qz + fmaf(rz, yl, fmaf(rz, yh, -qz));
}

// The same unit vector (bit for bit) together with what its rounding and
// the rounding of the pair distance left out, for the first-order energy
// correction of the partial-force pass:
//   u_res  r / |r| - u (the rounding residual of each component),
//   dres   |r| - sqrtf(d2), d2 the distance square the descriptor pass used,
//   inv    1 / |r| (FP32).
__host__ __device__ __forceinline__ void unit_vector_res(float rx, float ry, float rz, float d, float& ux,
                                                         float& uy, float& uz, float (&u_res)[3], float& dres,
                                                         float& inv)
{
    const float px = rx * rx, py = ry * ry, pz = rz * rz;
    const float ex = fmaf(rx, rx, -px), ey = fmaf(ry, ry, -py), ez = fmaf(rz, rz, -pz);
    float s1, t1, sh, t2;
    two_sum(px, py, s1, t1);
    two_sum(s1, pz, sh, t2);
    const float sl = ((t1 + t2) + (ex + ey)) + ez;
    const float y0 = 1.f / sqrtf(sh);
    const float a = sh * y0, ae = fmaf(sh, y0, -a);
    const float b = a * y0, be = fmaf(a, y0, -b);
    const float res = fmaf(-ae, y0, (1.f - b) - be) - sl * y0 * y0;
    const float yh = fmaf(0.5f * y0, res, y0);
    const float yl = fmaf(0.5f * y0, res, y0 - yh);
    const float qx = rx * yh, qy = ry * yh, qz = rz * yh;
    const float cx = fmaf(rx, yl, fmaf(rx, yh, -qx));
    const float cy = fmaf(ry, yl, fmaf(ry, yh, -qy));
    const float cz = fmaf(rz, yl, fmaf(rz, yh, -qz));
    ux = qx + cx;
    uy = qy + cy;
    uz = qz + cz;
    // |cx| <= ulp-scale of |qx|, so (qx - ux) is exact (Fast2Sum)
    u_res[0] = (qx - ux) + cx;
    u_res[1] = (qy - uy) + cy;
    u_res[2] = (qz - uz) + cz;
    // |r| = (sh + sl) (yh + yl) = lh + ll to first order in the small parts
    const float lh = sh * yh;
    const float ll = fmaf(sh, yh, -lh) + fmaf(sh, yl, sl * yh);
    dres = (lh - d) + ll;
    inv = yh;
}

// Pass 1 of atom i: the descriptor vector q (Eqs. 12-13 through the harmonic
// sums) and the harmonic sums S_nlm themselves.  Every lane of a warp must
// call it (inactive lanes pass cnt = 0): the ranks are walked in step.
template <class D = DescSi>
__host__ __device__ __forceinline__ void site_descriptors(int i, int n, int cnt, const SlotTable& nbr,
                                                          const float* __restrict__ xh,
                                                          const float* __restrict__ xl, const Box& box,
                                                          const SiteParams& P, const float (&hi)[3],
                                                          const float (&li)[3], float zi, float (&q)[D::Ndes],
                                                          HarmT<D>& S)
{
    constexpr int kNR = D::NR, kNA = D::NA, kNA2 = D::NA2;
    // radial sums are compensated (Kahan): q_0 ~ 4 accumulates ~28 terms and
    // its plain FP32 rounding dominates the site-energy error budget
    float qR[kNR], qC[kNR];
#pragma unroll
    for (int a = 0; a < kNR; ++a) qR[a] = qC[a] = 0.f;
#pragma unroll
    for (int a = 0; a < kNA2; ++a)
#pragma unroll
        for (int b = 0; b < kLM; ++b) S[a][b] = make_float2(0.f, 0.f);

    // Slots are sorted by increasing distance (MD lists); walk the ranks
    // downwards so the largest (nearest) terms are added last, with all lanes
    // of a warp at the same rank.
#ifdef __CUDA_ARCH__
    const int kmax = __reduce_max_sync(0xffffffffu, cnt);
#else
    const int kmax = cnt;
#endif
    NbSlot nx;
    fetch_slot(nbr, xh, xl, n, kmax - 1, cnt, nx);
    for (int k = kmax - 1; k >= 0; --k) {
        const NbSlot cur = nx;
        fetch_slot(nbr, xh, xl, n, k - 1, cnt, nx);
        if (k >= cnt) continue;
        const int j = cur.v & 0xFFFFFF;
        float rx, ry, rz;
        pair_vector(i, j, cur.v >> 24, hi, li, cur.h, cur.l, box, rx, ry, rz);
        const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        const float w = pair_weight(P, zi, cur.z);
        if (d2 < P.rcR2) {
            const float d = sqrtf(d2);
            float g[kNR];
            radial_g<kNR>(d, P.rcR, P.inv_rcR, g, w);
#pragma unroll
            for (int a = 0; a < kNR; ++a) {
                const float y = g[a] - qC[a];
                const float t = qR[a] + y;
                qC[a] = (t - qR[a]) - y;
                qR[a] = t;
            }
        }
        if (d2 < P.rcA2) {
            const float d = sqrtf(d2);
            float g[kNA];
            radial_g<kNA>(d, P.rcA, P.inv_rcA, g, w);
            float2 g2[kNA2];
            pair_orders(g, g2);
            float ux, uy, uz;
            unit_vector(rx, ry, rz, ux, uy, uz);
            sh_pass1(ux, uy, uz, g2, S);
        }
    }

    // descriptor vector: q_nl = sum_m c_lm S_nlm^2 (compensated), n outer, l inner
#pragma unroll
    for (int a = 0; a < kNR; ++a) q[a] = qR[a] - qC[a];
#pragma unroll
    for (int a = 0; a < kNA; ++a) {
#pragma unroll
        for (int l = 0; l < kLmax; ++l) q[kNR + a * kLmax + l] = 0.f;
        float qc[kLmax] = {0.f, 0.f, 0.f, 0.f};  // Kahan compensation per l
#pragma unroll
        for (int m = 0; m < kLM; ++m) {
            const int v = kNR + a * kLmax + sh_l(m);
            const float y = fmaf(sh_c(m) * harm(S, a, m), harm(S, a, m), -qc[sh_l(m)]);
            const float t = q[v] + y;
            qc[sh_l(m)] = (t - q[v]) - y;
            q[v] = t;
        }
#pragma unroll
        for (int l = 0; l < kLmax; ++l) q[kNR + a * kLmax + l] -= qc[l];
    }
}

// Partial force dU_i/dr_ij of one pair r = r_ij (d2 = |r|^2 < max cutoff^2)
// from the atom's coefficients A_nlm = 2 c_lm G_nl S_nlm and G_n (Eqs.
// 23-25): radial G_n g_n' rhat, angular sum_nlm A_nlm grad(g_n Z_lm).
//
// It also returns dE, the first-order correction of the site energy for the
// roundings of this pair's geometry in the descriptor pass: there the
// descriptors were evaluated at the FP32 distance d = sqrtf(d2) and unit
// vector u (each rounded), from the pair vector r rounded from the exact
// r + r_lo.  With dU/dd (the radial coefficient below) and dU/du (the
// unprojected harmonic gradient V, Z_lm being polynomials in u),
//   dE = dU/dd (|r + r_lo| - d) + dU/du . ((r + r_lo)/|r + r_lo| - u),
// which removes those roundings from U_i to second order (~1e-14 relative).
template <class D, class ArrA, class ArrR>
__host__ __device__ __forceinline__ void pair_partial_force(const float (&r)[3], const float (&r_lo)[3], float d2,
                                                            float w, const SiteParams& P, const ArrA& A,
                                                            const ArrR& GR, float& px, float& py, float& pz,
                                                            float& dE)
{
    constexpr int kNR = D::NR, kNA = D::NA;
    const float d = sqrtf(d2);
    float ux, uy, uz, u_res[3], dres, inv;
    unit_vector_res(r[0], r[1], r[2], d, ux, uy, uz, u_res, dres, inv);
    float radial = 0.f;  // coefficient of rhat (dU/dd)
    float Vx = 0.f, Vy = 0.f, Vz = 0.f;
    // geometry residuals: r_lo along and across u
    const float ur = fmaf(ux, r_lo[0], fmaf(uy, r_lo[1], uz * r_lo[2]));
    const float dd = dres + ur;
    if (d2 < P.rcR2) {
        float2 gd[kNR];
        radial_gd<kNR>(d, P.rcR, P.inv_rcR, gd, w);
#pragma unroll
        for (int a = 0; a < kNR; ++a) radial = fmaf(GR[a], gd[a].y, radial);
    }
    float eu = 0.f;
    if (d2 < P.rcA2) {
        float2 gd[kNA];
        radial_gd<kNA>(d, P.rcA, P.inv_rcA, gd, w);
        float2 Vxy = make_float2(0.f, 0.f);
        sh_pass2(ux, uy, uz, A, gd, radial, Vxy, Vz);
        const float dux = fmaf(fmaf(-ux, ur, r_lo[0]), inv, u_res[0]);
        const float duy = fmaf(fmaf(-uy, ur, r_lo[1]), inv, u_res[1]);
        const float duz = fmaf(fmaf(-uz, ur, r_lo[2]), inv, u_res[2]);
        eu = fmaf(Vxy.x, dux, fmaf(Vxy.y, duy, Vz * duz));
        // tangential projection of V, divided by r
        const float uv = fmaf(ux, Vxy.x, fmaf(uy, Vxy.y, uz * Vz));
        Vx = (Vxy.x - uv * ux) * inv;
        Vy = (Vxy.y - uv * uy) * inv;
        Vz = (Vz - uv * uz) * inv;
    }
    dE = fmaf(radial, dd, eu);
    px = fmaf(radial, ux, Vx);
    py = fmaf(radial, uy, Vy);
    pz = fmaf(radial, uz, Vz);
}

// Pass 1 and the network of atom i: site energy (hi + lo) and the
// coefficients A (kNA x kLM, in place of the harmonic sums S) and GR.
template <class D = DescSi>
__host__ __device__ __forceinline__ void site_coefficients(int i, bool active, int n, int cnt, const SlotTable& nbr,
                                                           const float* __restrict__ xh,
                                                           const float* __restrict__ xl, const Box& box,
                                                           const SiteParams& P, HarmT<D>& S,
                                                           float (&GR)[D::NR], float& U_hi, float& U_lo)
{
    constexpr int kNR = D::NR, kNA = D::NA, kNdes = D::Ndes;
    float hi[3], li[3], zi = 1.f;
    if (active) {
        load_pos(xh, xl, n, i, hi, li);
        zi = load_z(xh, i);
    }
    float q[kNdes];
    site_descriptors<D>(i, n, cnt, nbr, xh, xl, box, P, hi, li, zi, q, S);

    float G[kNdes];
    network(P.w, P.n_neu, q, G, U_hi, U_lo);

    // A_nlm = 2 c_lm G_nl S_nlm (reuses S)
#pragma unroll
    for (int a = 0; a < kNA; ++a) {
#pragma unroll
        for (int m = 0; m < kLM; ++m) {
            harm(S, a, m) *= 2.f * sh_c(m) * G[kNR + a * kLmax + sh_l(m)];
        }
    }
#pragma unroll
    for (int a = 0; a < kNR; ++a) GR[a] = G[a];
}

// Everything atom i contributes in the first force pass, in one thread: site
// energy and the partial forces dU_i/dr_ij of its first cnt slots (written
// through `out` for slots within max(rc_R, rc_A); other slots are left
// untouched).
template <class D = DescSi>
__host__ __device__ __forceinline__ void site_partial_forces(int i, bool active, int n, int cnt,
                                                             const SlotTable& nbr, const float* __restrict__ xh,
                                                             const float* __restrict__ xl, const Box& box,
                                                             const SiteParams& P, const PfOut& out, float& U_hi,
                                                             float& U_lo)
{
    HarmT<D> S;
    float GR[D::NR];
    site_coefficients<D>(i, active, n, cnt, nbr, xh, xl, box, P, S, GR, U_hi, U_lo);
    float hi[3], li[3], zi = 1.f;
    if (active) {
        load_pos(xh, xl, n, i, hi, li);
        zi = load_z(xh, i);
    }

    const float rc2max = P.rcR2 > P.rcA2 ? P.rcR2 : P.rcA2;
    // pass 2: partial forces, and the first-order energy correction of the
    // pair geometry's roundings (summed in FP32: each term is ~1e-7 eV)
    float dU = 0.f;
    NbSlot nx;
    fetch_slot(nbr, xh, xl, n, 0, cnt, nx);
    for (int k = 0; k < cnt; ++k) {
        const NbSlot cur = nx;
        fetch_slot(nbr, xh, xl, n, k + 1, cnt, nx);
        const int j = cur.v & 0xFFFFFF;
        float r[3], r_lo[3];
        pair_vector_lo(i, j, cur.v >> 24, hi, li, cur.h, cur.l, box, r, r_lo);
        const float d2 = fmaf(r[0], r[0], fmaf(r[1], r[1], r[2] * r[2]));
        if (!(d2 < rc2max)) continue;
        float px, py, pz, dE;
        pair_partial_force<D>(r, r_lo, d2, pair_weight(P, zi, cur.z), P, S, GR, px, py, pz, dE);
        dU += dE;
        const int ko = nbr.orig ? (int)nbr.orig[(size_t)k * nbr.stride + nbr.idx] : k;
        float* p = out.base + (size_t)ko * out.slot_stride;
        p[0] = px;
        p[out.comp_stride] = py;
        p[2 * out.comp_stride] = pz;
    }
    U_lo += dU;
}

// Force and per-atom virial of atom i from the stored partial forces
// (pf[k][i] float4 records, see nep_internal.cuh):
//   F_i = sum_j (p_ij - p_ji),  W_i^{ab} = sum_j r_ij^a p_ji^b   (Eqs. 4-6).
// With `mask` (the site pass's in-cutoff slot bits, [3][n]) the slots
// outside the cutoff issue no loads at all; without it every slot is
// loaded and tested.
// Software-pipelined two slots deep: while slot k is summed, slot k+1's
// neighbour position and both partial-force records are in flight (their
// addresses came in one iteration earlier), and slot k+2's list and
// reverse entries are being loaded, so no gather waits on the load of its
// own address.  The sums run in slot order.
// count of leading zero bits of a nonzero word
__host__ __device__ __forceinline__ int clz32(unsigned x)
{
#ifdef __CUDA_ARCH__
    return __clz((int)x);
#else
    return __builtin_clz(x);
#endif
}

struct AsmSlot {
    int v;
    float h[3], l[3];
    float4 po, pq;
};

__host__ __device__ __forceinline__ void assemble_atom(int i, int n, int m_cap, float rc2max,
                                                       const int* __restrict__ count, const SlotTable& nbr,
                                                       const int* __restrict__ rev, const float* __restrict__ xh,
                                                       const float* __restrict__ xl, const Box& box,
                                                       const float* __restrict__ pf, float (&F)[3], float (&W)[9],
                                                       const unsigned* __restrict__ mask = nullptr)
{
    float hi[3], li[3];
    load_pos(xh, xl, n, i, hi, li);
    int cnt = imin(count[i], m_cap);
    unsigned mb[3] = {~0u, ~0u, ~0u};
    if (mask) {
        mb[0] = mask[i];
        mb[1] = mask[(size_t)n + i];
        mb[2] = mask[(size_t)2 * n + i];
        // the loop ends after the last kept slot
        cnt = mb[2] ? 96 - clz32(mb[2]) : mb[1] ? 64 - clz32(mb[1]) : mb[0] ? 32 - clz32(mb[0]) : 0;
    }
    auto kept = [&](int k) { return ((k < 32 ? mb[0] >> k : k < 64 ? mb[1] >> (k - 32) : mb[2] >> (k - 64)) & 1u) != 0u; };
#pragma unroll
    for (int a = 0; a < 3; ++a) F[a] = 0.f;
#pragma unroll
    for (int a = 0; a < 9; ++a) W[a] = 0.f;
    const float4* pf4 = reinterpret_cast<const float4*>(pf);
    // list value and reverse slot of slot k
    auto load_idx = [&](int k, int& v, int& kr) {
        if (k < cnt && kept(k)) {
            v = nbr.slots[(size_t)k * nbr.stride + nbr.idx];
            kr = NEP_LDG(rev + (size_t)k * n + i);
        }
    };
    // the gathers of slot k, given its list value and reverse slot
    auto load_data = [&](int k, int v, int kr, AsmSlot& d) {
        if (k < cnt && kept(k)) {
            const int j = v & 0xFFFFFF;
            d.v = v;
            load_pos(xh, xl, n, j, d.h, d.l);
            d.po = NEP_LDG(pf4 + (size_t)k * n + i);
            d.pq = NEP_LDG(pf4 + (size_t)kr * n + j);
        }
    };
    int v1 = 0, kr1 = 0, v2 = 0, kr2 = 0;
    load_idx(0, v1, kr1);
    load_idx(1, v2, kr2);
    AsmSlot nx;
    load_data(0, v1, kr1, nx);
    for (int k = 0; k < cnt; ++k) {
        const AsmSlot cur = nx;
        load_data(k + 1, v2, kr2, nx);
        load_idx(k + 2, v2, kr2);
        if (!kept(k)) continue;
        const int j = cur.v & 0xFFFFFF;
        float r[3];
        pair_vector(i, j, cur.v >> 24, hi, li, cur.h, cur.l, box, r[0], r[1], r[2]);
        const float d2 = fmaf(r[0], r[0], fmaf(r[1], r[1], r[2] * r[2]));
        if (!(d2 < rc2max)) continue;
        // own p_ij and the neighbour's p_ji: one 16-byte record each
        const float pji[3] = {cur.pq.x, cur.pq.y, cur.pq.z};
        F[0] += cur.po.x - pji[0];
        F[1] += cur.po.y - pji[1];
        F[2] += cur.po.z - pji[2];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) W[3 * a + b] = fmaf(r[a], pji[b], W[3 * a + b]);
    }
}

}  // namespace nep
