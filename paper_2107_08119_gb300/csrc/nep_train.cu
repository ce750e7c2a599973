// nep_train.cu -- SNES population evaluation on a training set (Sec. II.D).
//
// Training set: structures of uneven size concatenated into one set of atoms
// (the paper's "super-structure", Sec. II.E), each with its own orthorhombic
// periodic box.  nep_dataset_create precomputes everything that does not
// depend on the parameters z (once):
//   q_i             descriptors [N][32]
//   J_ij            per pair, the derivatives of atom i's descriptor with
//                   respect to r_ij (Eqs. 24-25), stored at i's own slot for
//                   j: radial part as g_n'(r)/r times the vector r_ij (8
//                   floats + vector), angular part 24 x 3
//   B_i             sum over i's own pairs of J_ij ([N][32][3])
// Per population member k the loss then needs only
//   U_ki, G_ki = dU/dq  (network, Eqs. 21-22)
//   p_kji = G_kj . J_ji = dU_kj / dr_ji                           (Eq. 23)
//   F_ki = G_ki . B_i - sum_j p_kji                                (Eqs. 4-5)
//   W_k  = sum_i sum_j r_ij (x) p_kji                              (Eq. 6)
// and the RMSEs of Eqs. 29-34.  Kernels per evaluation:
//   k_pack      z_pop -> member-innermost weight layout
//   k_mlp_f32   FP32 network per (atom pair, member): U [N][P] and
//               G [N][32][Pst] (member innermost, Pst = P rounded up to 4)
//   k_pop_tc    the same network as BF16 tensor-core GEMMs (nep_pop_tc.cu)
//   k_contract_owner  warp per atom j, two members per lane: p_kji for j's
//               pairs from G_j held in registers, stored at the reverse slot
//   k_contract  warp per atom i: F_i from its slots' p_kji, |F - F_tar|^2,
//               U and W summed per chunk of 32 atoms
//   k_loss      per member: per-structure sums in a fixed order, RMSEs
// SNES (Eqs. 35-39): k_gauss (Philox4x32-10 normals, z = m + s r), k_snes_update.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "nep_dataset.cuh"

namespace nep {
namespace {

constexpr int kDsCap = 192;      // neighbour capacity per atom while building (within r_c)
constexpr int kChunkAtoms = 32;       // atoms per contraction block (chunks never span structures)
constexpr int kContractThreads = 128;  // owner pass: 4 warps per block, one atom per warp at a time
constexpr int kReceiverThreads = 256;  // receiver pass: 8 warps per chunk of atoms
constexpr int kMaxPop = 64;

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

// ------------------------------------------------------------------ build
__global__ void k_ds_split(int N, const double* __restrict__ pos, const int* __restrict__ sid,
                           const Box* __restrict__ boxes, float* __restrict__ xh, float* __restrict__ xl)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Box b = boxes[sid[i]];
    double wx[3];
    for (int d = 0; d < 3; ++d) {
        const double L = b.L[d];
        double x = pos[(size_t)d * N + i];
        double w = x - L * floor(x / L);
        if (w >= L) w -= L;
        if (w < 0.0) w = 0.0;
        wx[d] = w;
    }
    store_pos(xh, xl, i, wx);
}

__global__ void k_ds_list(int N, const int* __restrict__ sid, const int* __restrict__ sstart,
                          const Box* __restrict__ boxes, const float* __restrict__ xh, const float* __restrict__ xl,
                          float rc2, float rcA2, int* __restrict__ tmp, int* __restrict__ cnt, int* __restrict__ cntA,
                          unsigned* err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int s = sid[i];
    const Box b = boxes[s];
    float hi[3], li[3];
    load_pos(xh, xl, N, i, hi, li);
    int c = 0, ca = 0;
    for (int j = sstart[s]; j < sstart[s + 1]; ++j) {
        float hj[3], lj[3];
        load_pos(xh, xl, N, j, hj, lj);
        for (int sx = -b.img[0]; sx <= b.img[0]; ++sx)
            for (int sy = -b.img[1]; sy <= b.img[1]; ++sy)
                for (int sz = -b.img[2]; sz <= b.img[2]; ++sz) {
                    const int code = image_code(sx, sy, sz);
                    if (j == i && code == kImgCenter) continue;
                    float rx, ry, rz;
                    pair_vector(i, j, code, hi, li, hj, lj, b, rx, ry, rz);
                    const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                    if (d2 < rc2) {
                        if (c < kDsCap) tmp[(size_t)i * kDsCap + c] = j | (code << 24);
                        ++c;
                        if (d2 < rcA2) ++ca;
                    }
                }
    }
    cnt[i] = c;
    cntA[i] = ca;
    if (c > kDsCap) atomicOr(err, kErrOverflow);
}

__global__ void k_ds_compact(int N, const int* __restrict__ tmp, const long long* __restrict__ pstart,
                             const long long* __restrict__ astart, const int* __restrict__ sid,
                             const Box* __restrict__ boxes, const float* __restrict__ xh, const float* __restrict__ xl,
                             float rcA2, int* __restrict__ pj, long long* __restrict__ aidx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Box b = boxes[sid[i]];
    float hi[3], li[3];
    load_pos(xh, xl, N, i, hi, li);
    const long long p0 = pstart[i], p1 = pstart[i + 1];
    long long a = astart[i];
    for (long long p = p0; p < p1; ++p) {
        const int v = tmp[(size_t)i * kDsCap + (p - p0)];
        pj[p] = v;
        const int j = v & 0xFFFFFF;
        float hj[3], lj[3];
        load_pos(xh, xl, N, j, hj, lj);
        float rx, ry, rz;
        pair_vector(i, j, v >> 24, hi, li, hj, lj, b, rx, ry, rz);
        const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        aidx[p] = d2 < rcA2 ? a++ : -1;
    }
}

__global__ void k_ds_reverse(int N, const long long* __restrict__ pstart, const int* __restrict__ pj,
                             long long* __restrict__ rev, unsigned* err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (long long p = pstart[i]; p < pstart[i + 1]; ++p) {
        const int v = pj[p];
        const int j = v & 0xFFFFFF;
        const int target = i | ((124 - (v >> 24)) << 24);
        long long found = -1;
        for (long long q = pstart[j]; q < pstart[j + 1]; ++q)
            if (pj[q] == target) {
                found = q;
                break;
            }
        if (found < 0) {
            atomicOr(err, kErrReverse);
            found = p;
        }
        rev[p] = found;
    }
}

// Descriptors of atom i and the Jacobians of its descriptor with respect to
// each of its pair vectors r_ij, scattered to the reverse slots.

__global__ void k_ds_site(int N, const int* __restrict__ sid, const Box* __restrict__ boxes,
                          const float* __restrict__ xh, const float* __restrict__ xl,
                          const long long* __restrict__ pstart, const int* __restrict__ pj,
                          const long long* __restrict__ aidx, float rcR2,
                          float rcA2, float rcR, float rcA, float inv_rcR, float inv_rcA, float* __restrict__ q_out,
                          float* __restrict__ B_out, PairRec* __restrict__ rec, float* __restrict__ ang)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Box b = boxes[sid[i]];
    float hi[3], li[3];
    load_pos(xh, xl, N, i, hi, li);
    float qR[kNR], qC[kNR];
    float S[kNA][kLM];
    for (int a = 0; a < kNR; ++a) qR[a] = qC[a] = 0.f;
    for (int a = 0; a < kNA; ++a)
        for (int m = 0; m < kLM; ++m) S[a][m] = 0.f;
    const long long p0 = pstart[i], p1 = pstart[i + 1];
    for (long long p = p0; p < p1; ++p) {
        const int v = pj[p];
        const int j = v & 0xFFFFFF;
        float hj[3], lj[3];
        load_pos(xh, xl, N, j, hj, lj);
        float rx, ry, rz;
        pair_vector(i, j, v >> 24, hi, li, hj, lj, b, rx, ry, rz);
        const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        const float d = sqrtf(d2);
        if (d2 < rcR2) {
            float g[kNR];
            radial_g<kNR>(d, rcR, inv_rcR, g);
            for (int a = 0; a < kNR; ++a) {
                const float y = g[a] - qC[a];
                const float t = qR[a] + y;
                qC[a] = (t - qR[a]) - y;
                qR[a] = t;
            }
        }
        if (d2 < rcA2) {
            float g[kNA];
            radial_g<kNA>(d, rcA, inv_rcA, g);
            const float inv = 1.f / d;
            sh_pass1(rx * inv, ry * inv, rz * inv, g, S);
        }
    }
    float q[kNdes];
    for (int a = 0; a < kNR; ++a) q[a] = qR[a] - qC[a];
    for (int a = 0; a < kNA; ++a)
        for (int l = 0; l < kLmax; ++l) {
            float s2 = 0.f;
            for (int m = 0; m < kLM; ++m)
                if (sh_l(m) == l) s2 = fmaf(sh_c(m) * S[a][m], S[a][m], s2);
            q[kNR + a * kLmax + l] = s2;
        }
    for (int v = 0; v < kNdes; ++v) q_out[(size_t)i * kNdes + v] = q[v];

    float B[kNdes][3];
    for (int v = 0; v < kNdes; ++v) B[v][0] = B[v][1] = B[v][2] = 0.f;
    for (long long p = p0; p < p1; ++p) {
        const int v = pj[p];
        const int j = v & 0xFFFFFF;
        float hj[3], lj[3];
        load_pos(xh, xl, N, j, hj, lj);
        float r[3];
        pair_vector(i, j, v >> 24, hi, li, hj, lj, b, r[0], r[1], r[2]);
        const float d2 = fmaf(r[0], r[0], fmaf(r[1], r[1], r[2] * r[2]));
        const float d = sqrtf(d2);
        const float inv = 1.f / d;
        PairRec pr;
        pr.r[0] = r[0];
        pr.r[1] = r[1];
        pr.r[2] = r[2];
        pr.pad = 0.f;
        for (int a = 0; a < kNR; ++a) pr.gd[a] = 0.f;
        if (d2 < rcR2) {
            float g[kNR], dg[kNR];
            radial_g_dg<kNR>(d, rcR, inv_rcR, g, dg);
            for (int a = 0; a < kNR; ++a) {
                pr.gd[a] = dg[a] * inv;
                for (int c = 0; c < 3; ++c) B[a][c] = fmaf(pr.gd[a], r[c], B[a][c]);
            }
        }
        rec[p] = pr;  // owner order: the contraction's owner pass streams i's records
        if (d2 < rcA2) {
            float g[kNA], dg[kNA];
            radial_g_dg<kNA>(d, rcA, inv_rcA, g, dg);
            const float u[3] = {r[0] * inv, r[1] * inv, r[2] * inv};
            float Y[kLM], dY[kLM][3];
            sh_eval(u[0], u[1], u[2], Y, dY);
            float J[kNA * kLmax][3];
            for (int t = 0; t < kNA * kLmax; ++t) J[t][0] = J[t][1] = J[t][2] = 0.f;
            for (int m = 0; m < kLM; ++m) {
                const float ud = u[0] * dY[m][0] + u[1] * dY[m][1] + u[2] * dY[m][2];
                float tg[3];
                for (int c = 0; c < 3; ++c) tg[c] = (dY[m][c] - ud * u[c]) * inv;
                const int l = sh_l(m);
                for (int a = 0; a < kNA; ++a) {
                    const float two_s = 2.f * sh_c(m) * S[a][m];
                    for (int c = 0; c < 3; ++c)
                        J[a * kLmax + l][c] = fmaf(two_s, fmaf(dg[a] * Y[m], u[c], g[a] * tg[c]), J[a * kLmax + l][c]);
                }
            }
            const long long ai = aidx[p];
            float* out = ang + (size_t)ai * (kNA * kLmax * 3);
            for (int t = 0; t < kNA * kLmax; ++t)
                for (int c = 0; c < 3; ++c) {
                    out[t * 3 + c] = J[t][c];
                    B[kNR + t][c] += J[t][c];
                }
        }
    }
    for (int v = 0; v < kNdes; ++v)
        for (int c = 0; c < 3; ++c) B_out[((size_t)i * kNdes + v) * 3 + c] = B[v][c];
}

// ------------------------------------------------------------------ evaluation
// z_pop [P][n_par] -> W1t [n_neu][32][P], b1t [n_neu][P], w2t [n_neu][P], b2t [P]
__global__ void k_pack(int P, int n_neu, const float* __restrict__ z, float* __restrict__ W1t,
                       float* __restrict__ b1t, float* __restrict__ w2t, float* __restrict__ b2t)
{
    const int n_par = (kNdes + 2) * n_neu + 1;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P * n_par) return;
    const int k = e / n_par, t = e % n_par;
    const float v = z[e];
    if (t < n_neu * kNdes)
        W1t[(size_t)t * P + k] = v;
    else if (t < n_neu * kNdes + n_neu)
        b1t[(size_t)(t - n_neu * kNdes) * P + k] = v;
    else if (t < n_neu * kNdes + 2 * n_neu)
        w2t[(size_t)(t - n_neu * kNdes - n_neu) * P + k] = v;
    else
        b2t[k] = v;
}

// FP32 network, two atoms per thread (each weight load feeds two FMAs):
// thread t -> atom pair a = t / P, member k = t % P.
__global__ void __launch_bounds__(256) k_mlp_f32(int N, int P, int Pst, int n_neu, const float* __restrict__ q,
                                                 const float* __restrict__ W1t, const float* __restrict__ b1t,
                                                 const float* __restrict__ w2t, const float* __restrict__ b2t,
                                                 float* __restrict__ G, double* __restrict__ U)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long a = t / P;
    const int k = (int)(t % P);
    const long long i0 = 2 * a;
    if (i0 >= N) return;
    const bool two = i0 + 1 < N;
    const long long i1 = two ? i0 + 1 : i0;
    float q0[kNdes], q1[kNdes], G0[kNdes], G1[kNdes];
#pragma unroll
    for (int v = 0; v < kNdes; ++v) {
        q0[v] = q[i0 * kNdes + v];
        q1[v] = q[i1 * kNdes + v];
        G0[v] = G1[v] = 0.f;
    }
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
    for (int mu = 0; mu < n_neu; ++mu) {
        const float* w = W1t + (size_t)mu * kNdes * P + k;
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int v = 0; v < kNdes; ++v) {
            const float wv = w[(size_t)v * P];
            a0 = fmaf(wv, q0[v], a0);
            a1 = fmaf(wv, q1[v], a1);
        }
        const float bb = b1t[(size_t)mu * P + k], ww = w2t[(size_t)mu * P + k];
        const float x0 = tanhf(a0 - bb), x1 = tanhf(a1 - bb);
        float tt, e;
        float p = ww * x0, ep = fmaf(ww, x0, -p);
        two_sum(s0, p, tt, e);
        s0 = tt;
        c0 += e + ep;
        p = ww * x1;
        ep = fmaf(ww, x1, -p);
        two_sum(s1, p, tt, e);
        s1 = tt;
        c1 += e + ep;
        const float d0 = ww * fmaf(-x0, x0, 1.f), d1 = ww * fmaf(-x1, x1, 1.f);
#pragma unroll
        for (int v = 0; v < kNdes; ++v) {
            const float wv = w[(size_t)v * P];
            G0[v] = fmaf(d0, wv, G0[v]);
            G1[v] = fmaf(d1, wv, G1[v]);
        }
    }
    const double b2 = (double)b2t[k];
    U[i0 * P + k] = (double)s0 + (double)c0 - b2;
#pragma unroll
    for (int v = 0; v < kNdes; ++v) G[(i0 * kNdes + v) * Pst + k] = G0[v];
    if (two) {
        U[i1 * P + k] = (double)s1 + (double)c1 - b2;
#pragma unroll
        for (int v = 0; v < kNdes; ++v) G[(i1 * kNdes + v) * Pst + k] = G1[v];
    }
}

// Contraction, pass 1 (owner side): one warp per atom j, lane l holding
// members 2l and 2l + 1.  The lane loads its members' G_j once (registers).
// j's Jacobian records are contiguous (owner order), so the warp stages them
// into shared memory 32 pairs at a time with coalesced 16-byte loads, all in
// flight together, and then forms p_kji = G_kj . J_ji pair by pair from
// shared memory (broadcast reads), storing it at the slot of the reverse pair
// (i -> j) so that pass 2 finds the partial forces acting on i in i's own
// slot order.  The owner's virial contribution sum_i r_ij (x) p_kji
// (r_ij = -r_ji) goes to W6[j][w][k].  No atomics: every value has one writer.
constexpr int kOwnerChunk = 32;                                     // pairs staged per round
constexpr int kRecFloats = (int)(sizeof(PairRec) / sizeof(float));  // 12
constexpr int kAngFloats = kNA * kLmax * 3;                         // 72
constexpr int kOwnerStage = kOwnerChunk * (kRecFloats + kAngFloats);  // floats per warp

__global__ void __launch_bounds__(kContractThreads) k_contract_owner(
    int N, int P, int Pst, const float* __restrict__ G, const float* __restrict__ B,
    const long long* __restrict__ pstart, const long long* __restrict__ rev, const PairRec* __restrict__ rec,
    const long long* __restrict__ aidx, const float* __restrict__ ang, float* __restrict__ pbuf,
    float* __restrict__ w6out, float* __restrict__ fown)
{
    extern __shared__ float4 s_stage4[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* s_rec = reinterpret_cast<float*>(s_stage4) + (size_t)warp * kOwnerStage;
    float* s_ang = s_rec + kOwnerChunk * kRecFloats;
    const int k0 = 2 * lane;
    const bool ld = k0 < Pst;  // Pst is even: the float2 at k0 is inside the row
    const int warps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int j = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); j < N; j += warps) {
        float2 g[kNdes];
        const float* Gj = G + (size_t)j * kNdes * Pst + k0;
#pragma unroll
        for (int v = 0; v < kNdes; ++v)
            g[v] = ld ? *reinterpret_cast<const float2*>(Gj + (size_t)v * Pst) : make_float2(0.f, 0.f);
        // own term G_j . B_j (B_j = sum of j's own Jacobians), for pass 2
        {
            const float4* B4 = reinterpret_cast<const float4*>(B + (size_t)j * kNdes * 3);
            float f[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
            for (int u = 0; u < kNdes * 3 / 12; ++u) {  // 4 descriptors (12 floats) per step
                const float4 b0 = B4[3 * u], b1 = B4[3 * u + 1], b2 = B4[3 * u + 2];
                const float bb[4][3] = {{b0.x, b0.y, b0.z}, {b0.w, b1.x, b1.y}, {b1.z, b1.w, b2.x},
                                        {b2.y, b2.z, b2.w}};
#pragma unroll
                for (int d = 0; d < 4; ++d)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        f[0][c] = fmaf(g[4 * u + d].x, bb[d][c], f[0][c]);
                        f[1][c] = fmaf(g[4 * u + d].y, bb[d][c], f[1][c]);
                    }
            }
            if (ld) {
                float* o = fown + (size_t)j * 3 * Pst + k0;
#pragma unroll
                for (int c = 0; c < 3; ++c) *reinterpret_cast<float2*>(o + (size_t)c * Pst) = make_float2(f[0][c], f[1][c]);
            }
        }
        float w6[2][6] = {{0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}};
        const long long pe = pstart[j + 1];
        for (long long q0 = pstart[j]; q0 < pe; q0 += kOwnerChunk) {
            const int nq = (int)min((long long)kOwnerChunk, pe - q0);
            // this chunk's angular records are the consecutive ones starting at
            // the first angular pair's index (owner order assigns them in turn)
            const long long my_ai = lane < nq ? aidx[q0 + lane] : -1;
            const long long my_rv = lane < nq ? rev[q0 + lane] : 0;
            const unsigned angmask = __ballot_sync(0xffffffffu, my_ai >= 0);
            const int na = __popc(angmask);
            const long long a0 = na ? __shfl_sync(0xffffffffu, my_ai, __ffs(angmask) - 1) : 0;
            // stage pair records and angular blocks (16-byte pieces, all lanes)
            const float4* rsrc = reinterpret_cast<const float4*>(rec + q0);
            for (int t = lane; t < nq * kRecFloats / 4; t += 32)
                reinterpret_cast<float4*>(s_rec)[t] = rsrc[t];
            const float4* asrc = reinterpret_cast<const float4*>(ang + (size_t)a0 * kAngFloats);
            for (int t = lane; t < na * kAngFloats / 4; t += 32)
                reinterpret_cast<float4*>(s_ang)[t] = asrc[t];
            __syncwarp();
            for (int t = 0; t < nq; ++t) {
                const float* pr = s_rec + t * kRecFloats;  // r_ji [0..2], g_n'/r [3..10]
                const long long ai = __shfl_sync(0xffffffffu, my_ai, t);
                const long long rq = __shfl_sync(0xffffffffu, my_rv, t);
                float cr0 = 0.f, cr1 = 0.f;
#pragma unroll
                for (int v = 0; v < kNR; ++v) {
                    cr0 = fmaf(g[v].x, pr[3 + v], cr0);
                    cr1 = fmaf(g[v].y, pr[3 + v], cr1);
                }
                const float r0 = pr[0], r1 = pr[1], r2 = pr[2];
                float pv[2][3] = {{cr0 * r0, cr0 * r1, cr0 * r2}, {cr1 * r0, cr1 * r1, cr1 * r2}};
                if (ai >= 0) {
                    const float* A = s_ang + (size_t)(ai - a0) * kAngFloats;
#pragma unroll
                    for (int d = 0; d < kNA * kLmax; ++d) {
                        const float2 gg = g[kNR + d];
                        const float ja0 = A[3 * d], ja1 = A[3 * d + 1], ja2 = A[3 * d + 2];
                        pv[0][0] = fmaf(gg.x, ja0, pv[0][0]);
                        pv[0][1] = fmaf(gg.x, ja1, pv[0][1]);
                        pv[0][2] = fmaf(gg.x, ja2, pv[0][2]);
                        pv[1][0] = fmaf(gg.y, ja0, pv[1][0]);
                        pv[1][1] = fmaf(gg.y, ja1, pv[1][1]);
                        pv[1][2] = fmaf(gg.y, ja2, pv[1][2]);
                    }
                }
                if (ld) {
                    float* o = pbuf + (size_t)rq * 3 * Pst + k0;
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        *reinterpret_cast<float2*>(o + (size_t)c * Pst) = make_float2(pv[0][c], pv[1][c]);
                }
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    w6[m][0] = fmaf(-r0, pv[m][0], w6[m][0]);  // xx
                    w6[m][1] = fmaf(-r1, pv[m][1], w6[m][1]);  // yy
                    w6[m][2] = fmaf(-r2, pv[m][2], w6[m][2]);  // zz
                    w6[m][3] = fmaf(-r0, pv[m][1], w6[m][3]);  // xy
                    w6[m][4] = fmaf(-r1, pv[m][2], w6[m][4]);  // yz
                    w6[m][5] = fmaf(-r2, pv[m][0], w6[m][5]);  // zx
                }
            }
            __syncwarp();  // the stage is refilled by the next chunk
        }
        if (ld) {
            float* o = w6out + (size_t)j * 6 * Pst + k0;
#pragma unroll
            for (int w = 0; w < 6; ++w) *reinterpret_cast<float2*>(o + (size_t)w * Pst) = make_float2(w6[0][w], w6[1][w]);
        }
    }
}

// Contraction, pass 2 (receiver side): one block (8 warps) per chunk of <=
// kChunkAtoms atoms of one structure; each warp takes every 8th atom i, lane l
// members 2l and 2l + 1: F_i = G_i . B_i (from pass 1) - sum over i's slots of
// the stored p_kji (coalesced float2 rows, in slot order).  Per chunk and member: sums of
// U, of |F - F_tar|^2 and of the six virial components, in a fixed order
// (atoms in order within a warp, then the warps in order).
__global__ void __launch_bounds__(kReceiverThreads, 3) k_contract(
    int N, int P, int Pst, const int* __restrict__ chunk_begin, const int* __restrict__ chunk_end,
    const double* __restrict__ U, const long long* __restrict__ pstart, const float* __restrict__ fown,
    const float* __restrict__ pbuf, const float* __restrict__ w6in, const float* __restrict__ f_tar,
    double* __restrict__ partials)
{
    constexpr int kWarps = kReceiverThreads / 32;
    __shared__ double red[kWarps][kMaxPop][8];
    const int c = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k0 = 2 * lane;
    const bool on0 = k0 < P, on1 = k0 + 1 < P;
    const bool ld = k0 < Pst;
    // per-lane running sums live in shared memory (this lane's slots only)
#pragma unroll
    for (int m = 0; m < 2; ++m)
        if (k0 + m < kMaxPop)
#pragma unroll
            for (int w = 0; w < 8; ++w) red[warp][k0 + m][w] = 0.0;
    const int end = chunk_end[c];
    for (int i = chunk_begin[c] + warp; i < end; i += kWarps) {
        float F[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        if (ld) {  // own term G_i . B_i from pass 1
            const float* o = fown + (size_t)i * 3 * Pst + k0;
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                const float2 x = *reinterpret_cast<const float2*>(o + (size_t)cc * Pst);
                F[0][cc] = x.x;
                F[1][cc] = x.y;
            }
        }
        const long long pe = pstart[i + 1];
#pragma unroll 4
        for (long long p = pstart[i]; p < pe; ++p) {
            if (!ld) continue;
            const float* o = pbuf + (size_t)p * 3 * Pst + k0;
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                const float2 x = *reinterpret_cast<const float2*>(o + (size_t)cc * Pst);
                F[0][cc] -= x.x;
                F[1][cc] -= x.y;
            }
        }
        const float tx = f_tar[(size_t)i * 3], ty = f_tar[(size_t)i * 3 + 1], tz = f_tar[(size_t)i * 3 + 2];
        const float* wi = w6in + (size_t)i * 6 * Pst + k0;
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            if (!(m == 0 ? on0 : on1)) continue;
            const float dx = F[m][0] - tx, dy = F[m][1] - ty, dz = F[m][2] - tz;
            double* r = red[warp][k0 + m];
            r[0] += U[(size_t)i * P + k0 + m];
            r[1] += (double)dx * dx + (double)dy * dy + (double)dz * dz;
#pragma unroll
            for (int w = 0; w < 6; ++w) r[2 + w] += (double)wi[(size_t)w * Pst + m];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < P * 8; e += blockDim.x) {
        const int k = e / 8, w = e % 8;
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < kWarps; ++q) t += red[q][k][w];
        partials[((size_t)c * P + k) * 8 + w] = t;
    }
}

// One block per member: per structure, the chunk sums (fixed order), then the
// RMSEs of Eqs. 30-32 with energy and virial per atom, and L1, L2 (Eqs. 33-34).
__global__ void k_loss(int P, int S, int n_par, int N, const int* __restrict__ s_chunk0,
                       const int* __restrict__ s_natoms, const double* __restrict__ partials,
                       const double* __restrict__ e_tar, const double* __restrict__ w_tar,
                       const float* __restrict__ z, double l_e, double l_f, double l_v, double l_1, double l_2,
                       double* __restrict__ loss)
{
    const int k = blockIdx.x;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // se, sf, sv, l1, l2
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int c = s_chunk0[s]; c < s_chunk0[s + 1]; ++c)
            for (int w = 0; w < 8; ++w) v[w] += partials[((size_t)c * P + k) * 8 + w];
        const double na = (double)s_natoms[s];
        const double de = (v[0] - e_tar[s]) / na;
        acc[0] += de * de;
        acc[1] += v[1];
        for (int w = 0; w < 6; ++w) {
            const double dv = (v[2 + w] - w_tar[(size_t)s * 6 + w]) / na;
            acc[2] += dv * dv;
        }
    }
    for (int p = threadIdx.x; p < n_par; p += blockDim.x) {
        const double zz = (double)z[(size_t)k * n_par + p];
        acc[3] += fabs(zz);
        acc[4] += zz * zz;
    }
    __shared__ double tot[5];
    block_sum_store<5>(acc, tot);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double Le = sqrt(tot[0] / S), Lf = sqrt(tot[1] / (3.0 * N)), Lv = sqrt(tot[2] / (6.0 * S));
        const double L1 = tot[3] / n_par, L2 = sqrt(tot[4] / n_par);
        double* out = loss + (size_t)k * 6;
        out[0] = l_e * Le + l_f * Lf + l_v * Lv + l_1 * L1 + l_2 * L2;
        out[1] = Le;
        out[2] = Lf;
        out[3] = Lv;
        out[4] = L1;
        out[5] = L2;
    }
}

// ------------------------------------------------------------------ SNES
// Philox4x32-10 (Salmon et al., SC'11) from its published definition.
__device__ __forceinline__ void philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                                       uint32_t (&o)[4])
{
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    o[0] = c0;
    o[1] = c1;
    o[2] = c2;
    o[3] = c3;
}

// Standard normals for elements e = 0..count-1 of stream (seed, gen): block
// e/4 uses counter {e/4, 0, gen, 0x4E4550} and key {seed lo, seed hi};
// u = (w + 1/2) 2^-32; lanes 0/1 (2/3) are the Box-Muller pair of (u0, u1)
// ((u2, u3)).  Also writes z = m + s (.) r for a population of n_par-vectors.
__global__ void k_gauss(long long count, int n_par, unsigned long long seed, unsigned gen,
                        const float* __restrict__ m, const float* __restrict__ s, float* __restrict__ r,
                        float* __restrict__ z)
{
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (4 * b >= count) return;
    uint32_t w[4];
    philox((uint32_t)b, 0u, gen, 0x4E4550u, (uint32_t)seed, (uint32_t)(seed >> 32), w);
    float g[4];
    for (int pr = 0; pr < 2; ++pr) {
        const double u0 = ((double)w[2 * pr] + 0.5) * (1.0 / 4294967296.0);
        const double u1 = ((double)w[2 * pr + 1] + 0.5) * (1.0 / 4294967296.0);
        // Box-Muller in FP64 (a few operations per draw), rounded once to FP32
        const double rad = sqrt(-2.0 * log(u0));
        double sn, cs;
        sincospi(2.0 * u1, &sn, &cs);
        g[2 * pr] = (float)(rad * cs);
        g[2 * pr + 1] = (float)(rad * sn);
    }
    for (int l = 0; l < 4; ++l) {
        const long long e = 4 * b + l;
        if (e < count) {
            r[e] = g[l];
            if (z) {
                const int p = (int)(e % n_par);
                z[e] = fmaf(s[p], g[l], m[p]);
            }
        }
    }
}

// z = m + s (.) r for given draws.
__global__ void k_make_pop(long long count, int n_par, const float* __restrict__ m, const float* __restrict__ s,
                           const float* __restrict__ r, float* __restrict__ z)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    const int p = (int)(e % n_par);
    z[e] = fmaf(s[p], r[e], m[p]);
}

// Rank the members by (loss, index), then the natural gradients (Eqs. 36-37)
// with the rank utilities `util` and the update of m with the pre-update s
// (Eq. 38), then s (Eq. 39).  Every block ranks the (few) members itself and
// updates its own slice of parameters.
__global__ void k_snes_update(int P, int n_par, const double* __restrict__ loss, const float* __restrict__ util,
                              const float* __restrict__ r, float* __restrict__ m, float* __restrict__ s, float eta_m,
                              float eta_s, int* __restrict__ order_out)
{
    __shared__ int order[kMaxPop];
    __shared__ float u[kMaxPop];
    const int t = threadIdx.x;
    if (t < P) {
        const double lk = loss[(size_t)t * 6];
        int rank = 0;
        for (int j = 0; j < P; ++j) {
            const double lj = loss[(size_t)j * 6];
            rank += (lj < lk || (lj == lk && j < t)) ? 1 : 0;
        }
        order[rank] = t;
        u[t] = util[t];
    }
    __syncthreads();
    if (order_out && blockIdx.x == 0 && t < P) order_out[t] = order[t];
    const int p = blockIdx.x * blockDim.x + t;
    if (p >= n_par) return;
    float gm = 0.f, gs = 0.f;
    for (int q = 0; q < P; ++q) {
        const float rv = r[(size_t)order[q] * n_par + p];
        gm = fmaf(u[q], rv, gm);
        gs = fmaf(u[q], fmaf(rv, rv, -1.f), gs);
    }
    const float sp = s[p];
    m[p] = fmaf(eta_m * sp, gm, m[p]);
    s[p] = sp * expf(0.5f * eta_s * gs);
}

}  // namespace
}  // namespace nep

using namespace nep;


struct snes_state {
    nep_model* m = nullptr;
    int P = 0, n_par = 0;
    unsigned long long seed = 0;
    unsigned gen = 0;
    float* mean = nullptr;
    float* sigma = nullptr;
    float* r = nullptr;
    float* z = nullptr;
    double* loss = nullptr;
    int* order = nullptr;
    float* util = nullptr;  // rank utilities u_1..u_P (a constant of P)
};

namespace {

template <class T>
int dalloc(T** p, size_t count, long long* bytes)
{
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        return NEP_ERR_OOM;
    }
    if (bytes) *bytes += (long long)(count * sizeof(T));
    return NEP_OK;
}

template <class T>
void dfree(T*& p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

// member stride of G: a multiple of 4 so that a tensor-core member group
// (4 members) is one aligned 16-byte store
inline int member_stride(int P) { return (P + 3) / 4 * 4; }

int ensure_pop(nep_dataset* ds, int P)
{
    if (P <= ds->pop_cap) return NEP_OK;
    dfree(ds->W1t);
    dfree(ds->b1t);
    dfree(ds->w2t);
    dfree(ds->b2t);
    dfree(ds->G);
    dfree(ds->U);
    dfree(ds->partials);
    dfree(ds->packed);
    dfree(ds->pbuf);
    dfree(ds->w6);
    dfree(ds->fown);
    ds->pop_cap = 0;
    const int nn = ds->m->hp.n_neu;
    int rc;
    if ((rc = dalloc(&ds->W1t, (size_t)nn * kNdes * P, nullptr)) || (rc = dalloc(&ds->b1t, (size_t)nn * P, nullptr)) ||
        (rc = dalloc(&ds->w2t, (size_t)nn * P, nullptr)) || (rc = dalloc(&ds->b2t, (size_t)P, nullptr)) ||
        (rc = dalloc(&ds->G, (size_t)ds->N * kNdes * member_stride(P), nullptr)) ||
        (rc = dalloc(&ds->U, (size_t)ds->N * P, nullptr)) ||
        (rc = dalloc(&ds->partials, (size_t)ds->n_chunks * P * 8, nullptr)) ||
        (rc = dalloc(&ds->packed, pop_tc_packed_bytes(P), nullptr)) ||
        (rc = dalloc(&ds->pbuf, (size_t)ds->n_pairs * 3 * member_stride(P), nullptr)) ||
        (rc = dalloc(&ds->w6, (size_t)ds->N * 6 * member_stride(P), nullptr)) ||
        (rc = dalloc(&ds->fown, (size_t)ds->N * 3 * member_stride(P), nullptr)))
        return rc;
    // members past P in the last group of G are never written: keep them zero
    rc = cuda_fail(cudaMemset(ds->G, 0, sizeof(float) * (size_t)ds->N * kNdes * member_stride(P)), "clear G");
    if (rc) return rc;
    ds->pop_cap = P;
    return NEP_OK;
}

int evaluate(nep_model* m, nep_dataset* ds, const float* z_pop, int P, int precision, const double* lambdas,
             double* loss, cudaStream_t st)
{
    if (precision != NEP_PREC_FP32 && precision != NEP_PREC_BF16) {
        set_error("snes_evaluate_population: unknown precision %d", precision);
        return NEP_ERR_ARG;
    }
    int rc = ensure_pop(ds, P);
    if (rc) return rc;
    const int nn = m->hp.n_neu, n_par = m->n_par, Pst = member_stride(P);
    k_pack<<<blocks_for((long long)P * n_par, 256), 256, 0, st>>>(P, nn, z_pop, ds->W1t, ds->b1t, ds->w2t, ds->b2t);
    if (precision == NEP_PREC_BF16) {
        if ((rc = launch_pop_tc(ds->N, P, Pst, nn, ds->q, ds->W1t, ds->b1t, ds->w2t, ds->b2t, ds->packed, ds->G,
                                ds->U, m->d_err, st)))
            return rc;
    } else {
        const long long pairs = (ds->N + 1) / 2;
        k_mlp_f32<<<blocks_for(pairs * P, 256), 256, 0, st>>>(ds->N, P, Pst, nn, ds->q, ds->W1t, ds->b1t, ds->w2t,
                                                              ds->b2t, ds->G, ds->U);
    }
    const size_t ostage = (size_t)(kContractThreads / 32) * kOwnerStage * sizeof(float);
    if ((rc = cuda_fail(cudaFuncSetAttribute(k_contract_owner, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)ostage),
                        "contraction shared memory")))
        return rc;
    k_contract_owner<<<std::min(blocks_for(ds->N, kContractThreads / 32), 152 * 16), kContractThreads, ostage, st>>>(
        ds->N, P, Pst, ds->G, ds->B, ds->pstart, ds->rev, ds->rec, ds->aidx, ds->ang, ds->pbuf, ds->w6, ds->fown);
    k_contract<<<ds->n_chunks, kReceiverThreads, 0, st>>>(ds->N, P, Pst, ds->chunk_begin, ds->chunk_end, ds->U,
                                                          ds->pstart, ds->fown, ds->pbuf, ds->w6, ds->f_tar,
                                                          ds->partials);
    const double lam[5] = {lambdas ? lambdas[0] : 1.0, lambdas ? lambdas[1] : 1.0, lambdas ? lambdas[2] : 1.0,
                           lambdas ? lambdas[3] : 0.05, lambdas ? lambdas[4] : 0.05};
    k_loss<<<P, 256, 0, st>>>(P, ds->S, n_par, ds->N, ds->s_chunk0, ds->s_natoms, ds->partials, ds->e_tar, ds->w_tar,
                              z_pop, lam[0], lam[1], lam[2], lam[3], lam[4], loss);
    return cuda_fail(cudaGetLastError(), "population evaluation kernels");
}

}  // namespace

extern "C" {

int nep_dataset_create(nep_model* m, int n_struct, const int* n_atoms, const double* boxes, const double* pos,
                       const double* e_tar, const double* f_tar, const double* w_tar, nep_dataset** out)
{
    if (!m || !n_atoms || !boxes || !pos || !e_tar || !f_tar || !w_tar || !out || n_struct < 1) {
        set_error("nep_dataset_create: NULL argument or no structures");
        return NEP_ERR_ARG;
    }
    *out = nullptr;
    long long Nl = 0;
    for (int s = 0; s < n_struct; ++s) {
        if (n_atoms[s] < 1) {
            set_error("nep_dataset_create: structure %d has no atoms", s);
            return NEP_ERR_ARG;
        }
        Nl += n_atoms[s];
    }
    if (Nl > kMaxAtoms) {
        set_error("nep_dataset_create: too many atoms");
        return NEP_ERR_ARG;
    }
    const int N = (int)Nl, S = n_struct;
    const double rmax = m->hp.rc_R > m->hp.rc_A ? m->hp.rc_R : m->hp.rc_A;
    std::vector<Box> hbox(S);
    for (int s = 0; s < S; ++s) {
        int rc = setup_box(boxes + 9 * s, rmax, hbox[s]);
        if (rc) return rc;
        hbox[s].nc[0] = hbox[s].nc[1] = hbox[s].nc[2] = 0;
    }
    std::vector<int> hsid(N), hsstart(S + 1), hnat(S), hchunk0(S + 1), hcb, hce;
    hsstart[0] = 0;
    for (int s = 0; s < S; ++s) {
        hsstart[s + 1] = hsstart[s] + n_atoms[s];
        hnat[s] = n_atoms[s];
        for (int i = hsstart[s]; i < hsstart[s + 1]; ++i) hsid[i] = s;
        hchunk0[s] = (int)hcb.size();
        for (int b = hsstart[s]; b < hsstart[s + 1]; b += kChunkAtoms) {
            hcb.push_back(b);
            hce.push_back(std::min(b + kChunkAtoms, hsstart[s + 1]));
        }
    }
    hchunk0[S] = (int)hcb.size();
    std::vector<double> hpos((size_t)3 * N);
    for (int i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d) hpos[(size_t)d * N + i] = pos[(size_t)3 * i + d];
    std::vector<float> hf((size_t)3 * N);
    for (size_t e = 0; e < hf.size(); ++e) hf[e] = (float)f_tar[e];

    nep_dataset* ds = new (std::nothrow) nep_dataset();
    if (!ds) {
        set_error("nep_dataset_create: host allocation failed");
        return NEP_ERR_OOM;
    }
    ds->m = m;
    ds->S = S;
    ds->N = N;
    ds->n_chunks = (int)hcb.size();
    long long* bytes = &ds->bytes;
    double* dpos = nullptr;
    float*& xh = ds->xh;
    float*& xl = ds->xl;
    int *tmp = nullptr, *cnt = nullptr, *cnta = nullptr;
    long long*& rev = ds->rev;
    int rc = NEP_OK;
    auto fail = [&](int code) {
        dfree(dpos);
        dfree(tmp);
        dfree(cnt);
        dfree(cnta);
        nep_dataset_destroy(ds);
        return code;
    };
    if ((rc = dalloc(&ds->boxes, S, bytes)) || (rc = dalloc(&ds->sid, N, bytes)) ||
        (rc = dalloc(&ds->sstart, S + 1, bytes)) || (rc = dalloc(&ds->s_natoms, S, bytes)) ||
        (rc = dalloc(&ds->s_chunk0, S + 1, bytes)) || (rc = dalloc(&ds->chunk_begin, ds->n_chunks, bytes)) ||
        (rc = dalloc(&ds->chunk_end, ds->n_chunks, bytes)) || (rc = dalloc(&ds->q, (size_t)N * kNdes, bytes)) ||
        (rc = dalloc(&ds->B, (size_t)N * kNdes * 3, bytes)) || (rc = dalloc(&ds->pstart, (size_t)N + 1, bytes)) ||
        (rc = dalloc(&ds->e_tar, S, bytes)) || (rc = dalloc(&ds->f_tar, (size_t)3 * N, bytes)) ||
        (rc = dalloc(&ds->w_tar, (size_t)6 * S, bytes)) || (rc = dalloc(&dpos, (size_t)3 * N, nullptr)) ||
        (rc = dalloc(&xh, (size_t)4 * N, nullptr)) || (rc = dalloc(&xl, (size_t)4 * N, nullptr)) ||
        (rc = dalloc(&tmp, (size_t)N * kDsCap, nullptr)) || (rc = dalloc(&cnt, N, nullptr)) ||
        (rc = dalloc(&cnta, N, nullptr)))
        return fail(rc);
    cudaError_t e = cudaSuccess;
    auto up = [&](void* dst, const void* src, size_t b) {
        if (e == cudaSuccess) e = cudaMemcpy(dst, src, b, cudaMemcpyHostToDevice);
    };
    up(ds->boxes, hbox.data(), sizeof(Box) * S);
    up(ds->sid, hsid.data(), sizeof(int) * N);
    up(ds->sstart, hsstart.data(), sizeof(int) * (S + 1));
    up(ds->s_natoms, hnat.data(), sizeof(int) * S);
    up(ds->s_chunk0, hchunk0.data(), sizeof(int) * (S + 1));

    up(ds->chunk_begin, hcb.data(), sizeof(int) * hcb.size());
    up(ds->chunk_end, hce.data(), sizeof(int) * hce.size());
    up(dpos, hpos.data(), sizeof(double) * hpos.size());
    up(ds->e_tar, e_tar, sizeof(double) * S);
    up(ds->f_tar, hf.data(), sizeof(float) * hf.size());
    up(ds->w_tar, w_tar, sizeof(double) * 6 * S);
    if (e != cudaSuccess) return fail(cuda_fail(e, "dataset upload"));

    const float rc2 = (float)(rmax * rmax), rcA2 = (float)(m->hp.rc_A * m->hp.rc_A);
    const float rcR2 = (float)(m->hp.rc_R * m->hp.rc_R);
    k_ds_split<<<blocks_for(N, 256), 256>>>(N, dpos, ds->sid, ds->boxes, xh, xl);
    k_ds_list<<<blocks_for(N, 128), 128>>>(N, ds->sid, ds->sstart, ds->boxes, xh, xl, rc2, rcA2, tmp, cnt, cnta,
                                           m->d_err);
    if ((rc = cuda_fail(cudaDeviceSynchronize(), "dataset neighbour search"))) return fail(rc);
    unsigned bits = 0;
    cudaMemcpy(&bits, m->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (bits) {
        cudaMemset(m->d_err, 0, sizeof(unsigned));
        return fail(status_from_bits(bits));
    }
    std::vector<int> hc(N), hca(N);
    cudaMemcpy(hc.data(), cnt, sizeof(int) * N, cudaMemcpyDeviceToHost);
    cudaMemcpy(hca.data(), cnta, sizeof(int) * N, cudaMemcpyDeviceToHost);
    std::vector<long long> hps(N + 1), has(N + 1);
    hps[0] = has[0] = 0;
    for (int i = 0; i < N; ++i) {
        hps[i + 1] = hps[i] + hc[i];
        has[i + 1] = has[i] + hca[i];
    }
    ds->n_pairs = hps[N];
    ds->n_ang = has[N];
    long long* dastart = nullptr;
    if ((rc = dalloc(&ds->pj, (size_t)ds->n_pairs, bytes)) || (rc = dalloc(&ds->aidx, (size_t)ds->n_pairs, bytes)) ||
        (rc = dalloc(&ds->rec, (size_t)ds->n_pairs, bytes)) ||
        (rc = dalloc(&ds->ang, (size_t)ds->n_ang * kNA * kLmax * 3, bytes)) ||
        (rc = dalloc(&rev, (size_t)ds->n_pairs, bytes)) || (rc = dalloc(&dastart, (size_t)N + 1, nullptr)))
        return fail(rc);
    up(ds->pstart, hps.data(), sizeof(long long) * (N + 1));
    up(dastart, has.data(), sizeof(long long) * (N + 1));
    if (e != cudaSuccess) {
        dfree(dastart);
        return fail(cuda_fail(e, "dataset upload"));
    }
    k_ds_compact<<<blocks_for(N, 128), 128>>>(N, tmp, ds->pstart, dastart, ds->sid, ds->boxes, xh, xl, rcA2, ds->pj,
                                              ds->aidx);
    k_ds_reverse<<<blocks_for(N, 128), 128>>>(N, ds->pstart, ds->pj, rev, m->d_err);
    k_ds_site<<<blocks_for(N, 64), 64>>>(N, ds->sid, ds->boxes, xh, xl, ds->pstart, ds->pj, ds->aidx, rcR2,
                                         rcA2, (float)m->hp.rc_R, (float)m->hp.rc_A, (float)(1.0 / m->hp.rc_R),
                                         (float)(1.0 / m->hp.rc_A), ds->q, ds->B,
                                         ds->rec, ds->ang);
    rc = cuda_fail(cudaDeviceSynchronize(), "dataset precompute");
    dfree(dastart);
    if (rc) return fail(rc);
    cudaMemcpy(&bits, m->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (bits) {
        cudaMemset(m->d_err, 0, sizeof(unsigned));
        return fail(status_from_bits(bits));
    }
    dfree(dpos);
    dfree(tmp);
    dfree(cnt);
    dfree(cnta);
    *out = ds;
    return NEP_OK;
}

int nep_dataset_destroy(nep_dataset* ds)
{
    if (!ds) return NEP_OK;
    cudaDeviceSynchronize();
    dfree(ds->boxes);
    dfree(ds->sid);
    dfree(ds->sstart);
    dfree(ds->s_natoms);
    dfree(ds->s_chunk0);
    dfree(ds->chunk_begin);
    dfree(ds->chunk_end);
    dfree(ds->q);
    dfree(ds->xh);
    dfree(ds->xl);
    dfree(ds->B);
    dfree(ds->pstart);
    dfree(ds->pj);
    dfree(ds->rev);
    dfree(ds->aidx);
    dfree(ds->rec);
    dfree(ds->ang);
    dfree(ds->e_tar);
    dfree(ds->f_tar);
    dfree(ds->w_tar);
    dfree(ds->W1t);
    dfree(ds->b1t);
    dfree(ds->w2t);
    dfree(ds->b2t);
    dfree(ds->G);
    dfree(ds->U);
    dfree(ds->partials);
    dfree(ds->packed);
    dfree(ds->pbuf);
    dfree(ds->w6);
    dfree(ds->fown);
    free_adjoint(ds->adj);
    delete ds;
    return NEP_OK;
}

int nep_dataset_info(const nep_dataset* ds, int* n_atoms, long long* n_pairs, long long* device_bytes)
{
    if (!ds) {
        set_error("nep_dataset_info: NULL handle");
        return NEP_ERR_ARG;
    }
    if (n_atoms) *n_atoms = ds->N;
    if (n_pairs) *n_pairs = ds->n_pairs;
    if (device_bytes) *device_bytes = ds->bytes;
    return NEP_OK;
}

int nep_dataset_descriptors(const nep_dataset* ds, float* q, void* stream)
{
    if (!ds || !q) {
        set_error("nep_dataset_descriptors: NULL argument");
        return NEP_ERR_ARG;
    }
    return cuda_fail(cudaMemcpyAsync(q, ds->q, sizeof(float) * (size_t)ds->N * kNdes, cudaMemcpyDeviceToDevice,
                                     (cudaStream_t)stream),
                     "copy descriptors");
}

int snes_evaluate_population(nep_model* m, nep_dataset* ds, const float* z_pop, int n_pop, int precision,
                             const double* lambdas, double* loss, void* stream)
{
    if (!m || !ds || ds->m != m || !z_pop || !loss || n_pop < 1 || n_pop > kMaxPop) {
        set_error("snes_evaluate_population: bad arguments (1 <= n_pop <= %d, dataset of this model)", kMaxPop);
        return NEP_ERR_ARG;
    }
    return evaluate(m, ds, z_pop, n_pop, precision, lambdas, loss, (cudaStream_t)stream);
}

int snes_create(nep_model* m, int n_pop, const float* mean0, const float* sigma0, unsigned long long seed,
                snes_state** out)
{
    if (!m || !mean0 || !sigma0 || !out || n_pop < 2 || n_pop > kMaxPop) {
        set_error("snes_create: bad arguments (2 <= n_pop <= %d)", kMaxPop);
        return NEP_ERR_ARG;
    }
    *out = nullptr;
    snes_state* st = new (std::nothrow) snes_state();
    if (!st) {
        set_error("snes_create: host allocation failed");
        return NEP_ERR_OOM;
    }
    st->m = m;
    st->P = n_pop;
    st->n_par = m->n_par;
    st->seed = seed;
    const size_t np = (size_t)m->n_par, tot = np * n_pop;
    int rc;
    if ((rc = dalloc(&st->mean, np, nullptr)) || (rc = dalloc(&st->sigma, np, nullptr)) ||
        (rc = dalloc(&st->r, tot, nullptr)) || (rc = dalloc(&st->z, tot, nullptr)) ||
        (rc = dalloc(&st->loss, (size_t)n_pop * 6, nullptr)) || (rc = dalloc(&st->order, (size_t)n_pop, nullptr)) ||
        (rc = dalloc(&st->util, (size_t)n_pop, nullptr))) {
        snes_destroy(st);
        return rc;
    }
    // rank utilities (standard NES rank shaping, Sec. II.D.2):
    // u_q = max(0, ln(P/2 + 1) - ln q) / sum_q' max(0, ln(P/2 + 1) - ln q') - 1/P
    std::vector<float> util(n_pop);
    {
        const double top = std::log(n_pop / 2.0 + 1.0);
        double sum = 0.0;
        for (int q = 1; q <= n_pop; ++q) sum += std::fmax(0.0, top - std::log((double)q));
        for (int q = 1; q <= n_pop; ++q)
            util[q - 1] = (float)(std::fmax(0.0, top - std::log((double)q)) / sum - 1.0 / n_pop);
    }
    cudaError_t e = cudaMemcpy(st->mean, mean0, sizeof(float) * np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(st->sigma, sigma0, sizeof(float) * np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(st->util, util.data(), sizeof(float) * n_pop, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        snes_destroy(st);
        return cuda_fail(e, "snes_create upload");
    }
    *out = st;
    return NEP_OK;
}

int snes_destroy(snes_state* st)
{
    if (!st) return NEP_OK;
    cudaDeviceSynchronize();
    dfree(st->mean);
    dfree(st->sigma);
    dfree(st->r);
    dfree(st->z);
    dfree(st->loss);
    dfree(st->order);
    dfree(st->util);
    delete st;
    return NEP_OK;
}

int snes_step(snes_state* st, nep_dataset* ds, int precision, const double* lambdas, const float* r_in,
              double* loss_out, void* stream)
{
    if (!st || !ds || ds->m != st->m) {
        set_error("snes_step: bad arguments");
        return NEP_ERR_ARG;
    }
    cudaStream_t cs = (cudaStream_t)stream;
    const long long tot = (long long)st->P * st->n_par;
    if (r_in) {
        int rc = cuda_fail(cudaMemcpyAsync(st->r, r_in, sizeof(float) * tot, cudaMemcpyDeviceToDevice, cs), "copy r");
        if (rc) return rc;
        k_make_pop<<<blocks_for(tot, 256), 256, 0, cs>>>(tot, st->n_par, st->mean, st->sigma, st->r, st->z);
    } else {
        k_gauss<<<blocks_for((tot + 3) / 4, 256), 256, 0, cs>>>(tot, st->n_par, st->seed, st->gen, st->mean,
                                                                st->sigma, st->r, st->z);
    }
    int rc = evaluate(st->m, ds, st->z, st->P, precision, lambdas, st->loss, cs);
    if (rc) return rc;
    const float eta_s = (float)((3.0 + std::log((double)st->n_par)) / (5.0 * std::sqrt((double)st->n_par)));
    k_snes_update<<<blocks_for(st->n_par, 128), 128, 0, cs>>>(st->P, st->n_par, st->loss, st->util, st->r, st->mean, st->sigma,
                                                               1.f, eta_s, st->order);
    if (loss_out) {
        rc = cuda_fail(cudaMemcpyAsync(loss_out, st->loss, sizeof(double) * st->P * 6, cudaMemcpyDeviceToDevice, cs),
                       "copy loss");
        if (rc) return rc;
    }
    ++st->gen;
    return cuda_fail(cudaGetLastError(), "snes step kernels");
}

int snes_get_state(snes_state* st, float* mean, float* sigma, float* r_last, int* order, void* stream)
{
    if (!st) {
        set_error("snes_get_state: NULL handle");
        return NEP_ERR_ARG;
    }
    cudaStream_t cs = (cudaStream_t)stream;
    const size_t np = (size_t)st->n_par;
    cudaError_t e = cudaSuccess;
    if (mean) e = cudaMemcpyAsync(mean, st->mean, sizeof(float) * np, cudaMemcpyDeviceToDevice, cs);
    if (e == cudaSuccess && sigma) e = cudaMemcpyAsync(sigma, st->sigma, sizeof(float) * np, cudaMemcpyDeviceToDevice, cs);
    if (e == cudaSuccess && r_last)
        e = cudaMemcpyAsync(r_last, st->r, sizeof(float) * np * st->P, cudaMemcpyDeviceToDevice, cs);
    if (e == cudaSuccess && order) e = cudaMemcpyAsync(order, st->order, sizeof(int) * st->P, cudaMemcpyDeviceToDevice, cs);
    return cuda_fail(e, "snes_get_state");
}

}  // extern "C"
